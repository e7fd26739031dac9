// Matrix-free encoding operators (Eq. 1-4, 13-15):
//   E_c = M F_pe A Psi F_ro C   and its adjoint,
// with C the coil multiply, F_ro the centred zero-padded readout DFT, Psi the
// wave phase exp(-i phi(t,y,z)), A the block-diagonal patch compression
// (one A_g per group, Eq. 13), F_pe the centred phase-encode DFT and M the
// sampled-line gather.
//
// Readout stage ("k1"): one block per (phase-encode row, coil chunk).  The
// zero-padded N_tx-point DFT of an N_x-point row is computed as os twiddled
// N_x-point FFTs in shared memory (t = os m + s); the wave phase and the
// centring signs are folded into one per-row table.  The FP32 forward kernel
// applies A_g with FFMA as each coil's spectrum becomes available, so the
// uncompressed hybrid data never leaves the SM.
//
// Phase-encode stage ("k2"): one block per 8-column slab of the hybrid
// matrix H[row][col]; FFT along y (and z in 3D), gather / scatter of the
// sampled lines, and for E_c^H E_c the fused mask-projection with the
// squared norm ||E_c p||^2 accumulated for CG.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kK1Threads = 256;

// post(t) = (-1)^{m + nx/2} exp(i pi s/os) exp(-i phi(t,y,z)) / sqrt(ntx),
// t = os m + s: the centring factor of the readout DFT times the wave PSF,
// from the separable tables post_y[y][t] (centring, 1/sqrt(ntx), y wave term)
// and post_z[z][t] (z wave term).
__device__ __forceinline__ float2 readout_post(const Geo& g, int t, int y, int z) {
  const float2 py = g.post_y[(size_t)y * g.ntx + t];
  if (g.nz == 1) return py;
  return cmul(py, g.post_z[(size_t)z * g.ntx + t]);
}

struct K1Smem {
  float2* a;
  float2* b;
  float2* post;
  float2* pre;
  float2* tw;
};

__device__ __forceinline__ K1Smem k1_smem_setup(const Geo& g, int row, float2* base) {
  K1Smem sm;
  sm.a = base;
  sm.b = base + g.ntx;
  sm.post = base + 2 * g.ntx;
  sm.pre = base + 3 * g.ntx;
  sm.tw = base + 4 * g.ntx;
  const int y = row % g.ny, z = row / g.ny;
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) sm.tw[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < g.ntx; i += blockDim.x) {
    sm.pre[i] = g.pre[i];
    sm.post[i] = readout_post(g, i, y, z);
  }
  __syncthreads();
  return sm;
}

// One coil's readout spectrum for one row: returns the buffer holding
// U[t] (natural order, PSF applied).  u = c_n * x on entry.
__device__ __forceinline__ float2* k1_readout_fwd(const Geo& g, const K1Smem& sm,
                                                  const float2* __restrict__ crow,
                                                  const float2* __restrict__ xrow) {
  const int nx = g.nx, os = g.os;
  for (int i = threadIdx.x; i < g.ntx; i += blockDim.x) {
    const int xx = i % nx;
    sm.a[i] = cmul(cmul(crow[xx], xrow[xx]), sm.pre[i]);
  }
  __syncthreads();
  float2* res = fft_batch<-1>(sm.a, sm.b, os, nx, g.fx, sm.tw, threadIdx.x, blockDim.x);
  float2* out = (res == sm.a) ? sm.b : sm.a;
  for (int i = threadIdx.x; i < g.ntx; i += blockDim.x) {
    const int s = i / nx, m = i - s * nx;
    const int t = m * os + s;
    out[t] = cmul(res[i], sm.post[t]);
  }
  __syncthreads();
  return out;
}

// Inverse readout of one coil: U[t] (natural order) in `sm.a` on entry is
// multiplied by conj(post) and scattered to [s][m] in sm.b by the caller;
// this performs the os inverse FFTs and returns the result buffer.
__device__ __forceinline__ float2* k1_readout_adj_fft(const Geo& g, const K1Smem& sm) {
  return fft_batch<+1>(sm.b, sm.a, g.os, g.nx, g.fx, sm.tw, threadIdx.x, blockDim.x);
}

// -------------------------------------------------------------------------
// Forward E_c readout stage, FP32: Hpart[chunk][row][col] = sum over the
// chunk's coils of A_{g(p)} (Psi F_ro (c_n x))_patch.
template <int MAXJ>
__global__ void __launch_bounds__(kK1Threads) k1_fwd_fp32(Geo g, const float2* __restrict__ x,
                                                          const float2* __restrict__ coil,
                                                          const float2* __restrict__ AT,
                                                          float2* __restrict__ Hpart, int cpc) {
  extern __shared__ float2 smem[];
  const int row = blockIdx.x, chunk = blockIdx.y;
  const K1Smem sm = k1_smem_setup(g, row, smem);
  const size_t L = (size_t)g.rows * g.nx;
  const float2* xrow = x + (size_t)row * g.nx;

  float2 acc[MAXJ];
  int tb[MAXJ], ab[MAXJ], st[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    acc[j] = make_float2(0.f, 0.f);
    const int o = threadIdx.x + j * kK1Threads;
    tb[j] = o < g.ntxc ? g.out_tbase[o] : 0;
    ab[j] = o < g.ntxc ? g.out_abase[o] : 0;
    st[j] = o < g.ntxc ? g.out_astride[o] : 0;
  }
  const int n0 = chunk * cpc;
  const int n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; ++n) {
    const float2* U = k1_readout_fwd(g, sm, coil + n * L + (size_t)row * g.nx, xrow);
    const int nw = n * g.w;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int o = threadIdx.x + j * kK1Threads;
      if (o < g.ntxc) {
        const float2* Ap = AT + ab[j] + (size_t)nw * st[j];
        for (int tau = 0; tau < g.w; ++tau) cfma(acc[j], __ldg(Ap + (size_t)tau * st[j]), U[tb[j] + tau]);
      }
    }
    __syncthreads();
  }
  float2* out = Hpart + ((size_t)chunk * g.rows + row) * g.ntxc;
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    const int o = threadIdx.x + j * kK1Threads;
    if (o < g.ntxc) out[o] = acc[j];
  }
}

// Adjoint readout stage, FP32: xpart[chunk][row][x] = sum over the chunk's
// coils of conj(c_n) F_ro^H Psi^H A^H H2[row].
template <int MAXX>
__global__ void __launch_bounds__(kK1Threads) k1_adj_fp32(Geo g, const float2* __restrict__ H2,
                                                          const float2* __restrict__ coil,
                                                          const float2* __restrict__ A,
                                                          float2* __restrict__ xpart, int cpc) {
  extern __shared__ float2 smem[];
  const int row = blockIdx.x, chunk = blockIdx.y;
  const K1Smem sm = k1_smem_setup(g, row, smem);
  float2* Hs = smem + 4 * g.ntx + g.nx;
  const float2* hrow = H2 + (size_t)row * g.ntxc;
  for (int i = threadIdx.x; i < g.ntxc; i += blockDim.x) Hs[i] = hrow[i];
  __syncthreads();
  const size_t L = (size_t)g.rows * g.nx;
  float2 xacc[MAXX];
#pragma unroll
  for (int j = 0; j < MAXX; ++j) xacc[j] = make_float2(0.f, 0.f);
  const int n0 = chunk * cpc;
  const int n1 = min(g.nc, n0 + cpc);
  const int nx = g.nx, os = g.os, w = g.w, ns = g.ns;
  for (int n = n0; n < n1; ++n) {
    // A^H: U[t] = sum_k conj(A_g[k][n w + tau]) H2[off_p + k]; A is [k][i]
    // so neighbouring t (neighbouring tau) read neighbouring addresses.
    for (int t = threadIdx.x; t < g.ntx; t += blockDim.x) {
      const int p = t / w, tau = t - p * w;
      const int gg = g.pg[p];
      const int kg = g.keep[gg];
      const float2* Ap = A + g.aoff[gg] + n * w + tau;
      const float2* hp = Hs + g.poff[p];
      float2 v = make_float2(0.f, 0.f);
      for (int k = 0; k < kg; ++k) cfmac(v, __ldg(Ap + (size_t)k * ns), hp[k]);
      v = cmulc(sm.post[t], v);
      const int m = t / os, s = t - m * os;
      sm.b[s * nx + m] = v;
    }
    __syncthreads();
    float2* res = k1_readout_adj_fft(g, sm);
    const float2* crow = coil + n * L + (size_t)row * nx;
#pragma unroll
    for (int j = 0; j < MAXX; ++j) {
      const int xx = threadIdx.x + j * kK1Threads;
      if (xx < nx) {
        float2 u = make_float2(0.f, 0.f);
        for (int s = 0; s < os; ++s) cfmac(u, sm.pre[s * nx + xx], res[s * nx + xx]);
        cfmac(xacc[j], crow[xx], u);
      }
    }
    __syncthreads();
  }
  float2* out = xpart + ((size_t)chunk * g.rows + row) * nx;
#pragma unroll
  for (int j = 0; j < MAXX; ++j) {
    const int xx = threadIdx.x + j * kK1Threads;
    if (xx < nx) out[xx] = xacc[j];
  }
}

// ------------------------------------------------------------------ launchers --

cudaError_t launch_k1_fwd_fp32(const Geo& g, const float2* x, const float2* coil, const float2* AT,
                               float2* Hpart, int nchunk, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  dim3 grid(g.rows, nchunk);
  const size_t sm = k1_smem_bytes(g);
  const int need = (g.ntxc + kK1Threads - 1) / kK1Threads;
#define K1F(J)                                                                               \
  {                                                                                          \
    cudaFuncSetAttribute(k1_fwd_fp32<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    note_launches(1); k1_fwd_fp32<J><<<grid, kK1Threads, sm, st>>>(g, x, coil, AT, Hpart, cpc);                \
    return cudaGetLastError();                                                               \
  }
  if (need <= 2) K1F(2)
  if (need <= 4) K1F(4)
  if (need <= 8) K1F(8)
  if (need <= 16) K1F(16)
  if (need <= 24) K1F(24)
  if (need <= 32) K1F(32)
#undef K1F
  return cudaErrorInvalidValue;
}

cudaError_t launch_k1_adj_fp32(const Geo& g, const float2* H2, const float2* coil, const float2* A,
                               float2* xpart, int nchunk, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  dim3 grid(g.rows, nchunk);
  const size_t sm = k1_smem_bytes(g) + sizeof(float2) * (size_t)g.ntxc;
  const int need = (g.nx + kK1Threads - 1) / kK1Threads;
#define K1A(J)                                                                               \
  {                                                                                          \
    cudaFuncSetAttribute(k1_adj_fp32<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    note_launches(1); k1_adj_fp32<J><<<grid, kK1Threads, sm, st>>>(g, H2, coil, A, xpart, cpc);               \
    return cudaGetLastError();                                                               \
  }
  if (need <= 1) K1A(1)
  if (need <= 2) K1A(2)
#undef K1A
  return cudaErrorInvalidValue;
}

}  // namespace gpjc
