// Nonlinear local-B0 modulation (Sec. 2.1-2.2, Eq. 2-3, Eq. 14): the
// modulation phase phi(t, r) = sum_l a_l(t) B_l(r) of local B0 coils depends
// on the readout position x, so the readout is no longer a DFT and each
// phase-encode row (y, z) has its own compressed readout encoding matrix
//   G_row[off_p + k][x] = sum_{n, tau} A_{g(p)}[k][n w + tau] c_n(z, y, x)
//                          exp(-i [2 pi t_c x_c / N_tx + phi(p w + tau, z, y, x)]) / sqrt(N_tx),
// stored in HBM ([row][N'_tx][N_x] complex64, the per-column matrices the
// paper stores) and applied as a batched matrix-vector product; the
// phase-encode DFT still factors out (phi does not depend on the phase-encode
// step), so the phase-encode stage of the wave operator serves unchanged.
//
// Build: one block per (patch, row); the block generates the uncompressed
// encoding block E[n w + tau][x] of its patch for a tile of x in shared
// memory (the readout phase from the exact integer product t_c x_c mod N_tx,
// the local-B0 phase from the fields in FP32) and contracts it with A_g.
// Apply: G is streamed from HBM once per application (HBM-bound,
// 8 N'_tx N_x bytes per row): forward one warp per output column with
// 16-byte loads along x, adjoint threads over x pairs and column subsets
// with the compressed row staged in shared memory, partial images per
// column chunk.
#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kLbThreads = 256;

__global__ void __launch_bounds__(kLbThreads) k_lb0_build(Geo g, int nfields, int tx, const float2* __restrict__ coil,
                                                         const float* __restrict__ fields,
                                                         const float* __restrict__ amps,
                                                         const float2* __restrict__ A, float2* __restrict__ G) {
  extern __shared__ __align__(16) float2 er[];  // [ns][tx]
  const int p = blockIdx.x, row = blockIdx.y;
  const int grp = g.pg[p], keep = g.keep[grp];
  const float2* Ag = A + g.aoff[grp];  // [keep][ns]
  const int nx = g.nx, w = g.w, ns = g.ns, ntx = g.ntx;
  const size_t L = (size_t)g.rows * nx;
  const float inv = g.inv_sqrt_ntx;
  float2* Gout = G + ((size_t)row * g.ntxc + g.poff[p]) * nx;
  for (int x0 = 0; x0 < nx; x0 += tx) {
    for (int idx = threadIdx.x; idx < ns * tx; idx += blockDim.x) {
      const int i = idx / tx, xl = idx - i * tx, x = x0 + xl;
      float2 e = make_float2(0.f, 0.f);
      if (x < nx) {
        const int n = i / w, tau = i - n * w, t = p * w + tau;
        // readout phase 2 pi (t_c x_c mod N_tx) / N_tx, exact reduction
        long long m = (long long)(t - ntx / 2) * (long long)(x - nx / 2);
        m %= ntx;
        if (m < 0) m += ntx;
        float s1, c1;
        sincospif(-2.0f * (float)m / (float)ntx, &s1, &c1);
        float ph = 0.f;
        for (int l = 0; l < nfields; ++l) ph = fmaf(amps[(size_t)l * ntx + t], fields[(size_t)l * L + (size_t)row * nx + x], ph);
        float s2, c2;
        sincosf(-ph, &s2, &c2);
        const float2 ex = make_float2(c1 * c2 - s1 * s2, c1 * s2 + s1 * c2);
        const float2 cv = coil[(size_t)n * L + (size_t)row * nx + x];
        e = cscale(cmul(cv, ex), inv);
      }
      er[idx] = e;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < keep * tx; o += blockDim.x) {
      const int k = o / tx, xl = o - k * tx, x = x0 + xl;
      const float2* a = Ag + (size_t)k * ns;
      float2 acc = make_float2(0.f, 0.f);
      for (int i = 0; i < ns; ++i) cfma(acc, __ldg(a + i), er[i * tx + xl]);
      if (x < nx) Gout[(size_t)k * nx + x] = acc;
    }
    __syncthreads();
  }
}

// H[row][j] = sum_x G[row][j][x] x[row][x]: one warp per column j, x in pairs
// (16-byte loads; nx is even)
constexpr int kLbJPerWarp = 4;
__global__ void __launch_bounds__(kLbThreads) k_lb0_fwd(int nx, int ntxc, const float2* __restrict__ G,
                                                       const float2* __restrict__ x, float2* __restrict__ H) {
  extern __shared__ __align__(16) float2 xs[];  // [nx]
  const int row = blockIdx.y;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) xs[i] = x[(size_t)row * nx + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int j0 = (blockIdx.x * nw + warp) * kLbJPerWarp;
  const int half = nx >> 1;
  const float4* xs4 = reinterpret_cast<const float4*>(xs);
#pragma unroll
  for (int jj = 0; jj < kLbJPerWarp; ++jj) {
    const int j = j0 + jj;
    if (j >= ntxc) break;
    const float4* gr = reinterpret_cast<const float4*>(G + ((size_t)row * ntxc + j) * nx);
    float2 acc = make_float2(0.f, 0.f);
    for (int q = lane; q < half; q += 32) {
      const float4 gv = __ldcs(gr + q);  // streamed once per application
      const float4 xv = xs4[q];
      cfma(acc, make_float2(gv.x, gv.y), make_float2(xv.x, xv.y));
      cfma(acc, make_float2(gv.z, gv.w), make_float2(xv.z, xv.w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) H[(size_t)row * ntxc + j] = acc;
  }
}

// xpart[c][row][x] = sum_{j in chunk c} conj(G[row][j][x]) H2[row][j]:
// threads = (x pair q, column subset s) with nx / 2 <= 256 pairs (the plan
// caps nx at 512), so one pass covers the row; the chunk's H2 entries sit in
// shared memory and the subsets' sums are added in a fixed order
__global__ void __launch_bounds__(kLbThreads) k_lb0_adj(int nx, int ntxc, int rows, int jper,
                                                       const float2* __restrict__ G, const float2* __restrict__ H2,
                                                       float2* __restrict__ xpart) {
  extern __shared__ __align__(16) float2 hs[];  // [jper], then [nsub][half][2] partial sums
  const int c = blockIdx.x, row = blockIdx.y;
  const int j0 = c * jper, j1 = min(ntxc, j0 + jper);
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) hs[j - j0] = H2[(size_t)row * ntxc + j];
  __syncthreads();
  const int half = nx >> 1;
  const int nsub = (int)blockDim.x / half;
  const int q = threadIdx.x % half, s = threadIdx.x / half;
  float2* red = hs + jper;
  if (s < nsub) {
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    const float4* g4 = reinterpret_cast<const float4*>(G + (size_t)row * ntxc * nx) + q;
    int j = j0 + s;
    // four independent 16-byte loads in flight per thread
    for (; j + 3 * nsub < j1; j += 4 * nsub) {
      float4 gv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) gv[u] = __ldcs(g4 + (size_t)(j + u * nsub) * half);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 h = hs[j + u * nsub - j0];
        cfmac(a0, make_float2(gv[u].x, gv[u].y), h);
        cfmac(a1, make_float2(gv[u].z, gv[u].w), h);
      }
    }
    for (; j < j1; j += nsub) {
      const float4 gv = __ldcs(g4 + (size_t)j * half);
      const float2 h = hs[j - j0];
      cfmac(a0, make_float2(gv.x, gv.y), h);
      cfmac(a1, make_float2(gv.z, gv.w), h);
    }
    red[2 * (s * half + q)] = a0;
    red[2 * (s * half + q) + 1] = a1;
  }
  __syncthreads();
  if (threadIdx.x < half) {
    float2 r0 = make_float2(0.f, 0.f), r1 = make_float2(0.f, 0.f);
    for (int k = 0; k < nsub; ++k) {
      r0 = cadd(r0, red[2 * (k * half + threadIdx.x)]);
      r1 = cadd(r1, red[2 * (k * half + threadIdx.x) + 1]);
    }
    float2* out = xpart + ((size_t)c * rows + row) * nx + 2 * threadIdx.x;
    out[0] = r0;
    out[1] = r1;
  }
}

// ------------------------------------------------------------------ host side --
// x tile of the build: the largest power of two <= 32 whose encoding tile
// [ns][tx] fits in 200 KB of shared memory (0 when even tx = 1 does not)
int lb0_build_tile(int ns) {
  int tx = 32;
  while (tx > 0 && (size_t)ns * tx * sizeof(float2) > (size_t)200 * 1024) tx >>= 1;
  return tx;
}

cudaError_t launch_lb0_build(const Geo& g, int nfields, const float2* coil, const float* fields, const float* amps,
                             const float2* A, float2* G, cudaStream_t st) {
  const int tx = lb0_build_tile(g.ns);
  if (tx < 1) return cudaErrorInvalidValue;
  const size_t sm = (size_t)g.ns * tx * sizeof(float2);
  cudaFuncSetAttribute(k_lb0_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k_lb0_build<<<dim3(g.np, g.rows), kLbThreads, sm, st>>>(g, nfields, tx, coil, fields, amps, A, G);
  return cudaGetLastError();
}

cudaError_t launch_lb0_fwd(const Geo& g, const float2* G, const float2* x, float2* H, cudaStream_t st) {
  const int per_block = (kLbThreads / 32) * kLbJPerWarp;
  const dim3 grid((g.ntxc + per_block - 1) / per_block, g.rows);
  note_launches(1); k_lb0_fwd<<<grid, kLbThreads, sizeof(float2) * g.nx, st>>>(g.nx, g.ntxc, G, x, H);
  return cudaGetLastError();
}

cudaError_t launch_lb0_adj(const Geo& g, const float2* G, const float2* H2, float2* xpart, int nsplit, cudaStream_t st) {
  const int jper = (g.ntxc + nsplit - 1) / nsplit;
  const size_t sm = sizeof(float2) * ((size_t)jper + 2 * (size_t)kLbThreads);
  cudaFuncSetAttribute(k_lb0_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k_lb0_adj<<<dim3(nsplit, g.rows), kLbThreads, sm, st>>>(g.nx, g.ntxc, g.rows, jper, G, H2, xpart);
  return cudaGetLastError();
}

}  // namespace gpjc
