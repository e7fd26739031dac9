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
// Phase-encode stage ("k2"): one block per 16-column slab of the hybrid
// matrix H[row][col]; FFT along y (and z in 3D), gather / scatter of the
// sampled lines, and for E_c^H E_c the fused mask-projection with the
// squared norm ||E_c p||^2 accumulated for CG.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kK1Threads = 256;
constexpr int kK2Threads = 256;
constexpr int kCB = 16;  // columns per phase-encode block

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

// -------------------------------------------------------------------------
// Phase-encode stage.  H is [rows][ncols]; a block owns kCB columns.
// Centred unitary DFT along y: F[ky,y] = (-1)^{y} (-1)^{ky + ny/2}
// exp(-2 pi i ky y / ny) / sqrt(ny).

__device__ __forceinline__ float sgn(int k) { return (k & 1) ? -1.0f : 1.0f; }

// 2D forward: Sc[l][col] = (F_y sum_chunk Hpart)[ky_l][col]
__global__ void __launch_bounds__(kK2Threads) k2_fwd_2d(Geo g, const float2* __restrict__ Hpart,
                                                        int nchunk, int ncols,
                                                        float2* __restrict__ Sc) {
  extern __shared__ float2 smem[];
  const int ny = g.ny, bs = ny + 1;
  float2* a = smem;
  float2* b = smem + kCB * bs;
  float2* tw = smem + 2 * kCB * bs;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = g.tw_y[i];
  const int col0 = blockIdx.x * kCB;
  const size_t plane = (size_t)g.rows * ncols;
  for (int i = threadIdx.x; i < ny * kCB; i += blockDim.x) {
    const int y = i / kCB, c = i - y * kCB;
    const int col = col0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (col < ncols)
      for (int ch = 0; ch < nchunk; ++ch) v = cadd(v, Hpart[ch * plane + (size_t)y * ncols + col]);
    a[c * bs + y] = cscale(v, sgn(y));
  }
  __syncthreads();
  float2* res = fft_batch<-1>(a, b, kCB, bs, g.fy, tw, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < g.n_lines * kCB; i += blockDim.x) {
    const int l = i / kCB, c = i - l * kCB;
    const int col = col0 + c;
    if (col < ncols) {
      const int ky = g.line_ky[l];
      Sc[(size_t)l * ncols + col] = cscale(res[c * bs + ky], sgn(ky + ny / 2) * g.inv_sqrt_ny);
    }
  }
}

// 2D adjoint: H[y][col] = (F_y^H M^T Sc)[y][col]
__global__ void __launch_bounds__(kK2Threads) k2_adj_2d(Geo g, const float2* __restrict__ Sc, int ncols,
                                                        float2* __restrict__ H) {
  extern __shared__ float2 smem[];
  pe_adj2d_body(g, Sc, ncols, H, blockIdx.x, smem);
}

// 2D normal: H2 = F_y^H M^T M F_y (sum_chunk Hpart); ||M F_y H||^2 reduced
// into *qq (deterministic grid sum).
__global__ void __launch_bounds__(kK2Threads) k2_normal_2d(Geo g, const float2* __restrict__ Hpart,
                                                           int nchunk, int ncols,
                                                           float2* __restrict__ H2, double* partials,
                                                           unsigned* counter, double* qq) {
  extern __shared__ float2 smem[];
  __shared__ double red[32];
  const double tot = pe_normal2d_body<false>(g, Hpart, nchunk, ncols, H2, blockIdx.x, smem);
  // the block total is valid in thread 0 only
  if (qq) grid_sum_finalize(threadIdx.x == 0 ? tot : 0.0, partials, counter, qq, red);
}

// ---- 3D: y pass over (z, column slab), z pass over (ky, column slab).
// T[z][ky][col] = F_y (sum_chunk Hpart)[z][.][col]
__global__ void __launch_bounds__(kK2Threads) k2_y_fwd3d(Geo g, const float2* __restrict__ Hpart,
                                                         int nchunk, int ncols, float2* __restrict__ T) {
  extern __shared__ float2 smem[];
  const int ny = g.ny, bs = ny + 1, z = blockIdx.y;
  float2* a = smem;
  float2* b = smem + kCB * bs;
  float2* tw = smem + 2 * kCB * bs;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = g.tw_y[i];
  const int col0 = blockIdx.x * kCB;
  const size_t plane = (size_t)g.rows * ncols;
  for (int i = threadIdx.x; i < ny * kCB; i += blockDim.x) {
    const int y = i / kCB, c = i - y * kCB;
    const int col = col0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (col < ncols) {
      const size_t idx = ((size_t)z * ny + y) * ncols + col;
      for (int ch = 0; ch < nchunk; ++ch) v = cadd(v, Hpart[ch * plane + idx]);
    }
    a[c * bs + y] = cscale(v, sgn(y));
  }
  __syncthreads();
  float2* res = fft_batch<-1>(a, b, kCB, bs, g.fy, tw, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < ny * kCB; i += blockDim.x) {
    const int ky = i / kCB, c = i - ky * kCB;
    const int col = col0 + c;
    if (col < ncols)
      T[((size_t)z * ny + ky) * ncols + col] = cscale(res[c * bs + ky], sgn(ky + ny / 2) * g.inv_sqrt_ny);
  }
}

// H[z][y][col] = F_y^H T[z][.][col]
__global__ void __launch_bounds__(kK2Threads) k2_y_adj3d(Geo g, const float2* __restrict__ T, int ncols,
                                                         float2* __restrict__ H) {
  extern __shared__ float2 smem[];
  const int ny = g.ny, bs = ny + 1, z = blockIdx.y;
  float2* a = smem;
  float2* b = smem + kCB * bs;
  float2* tw = smem + 2 * kCB * bs;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = g.tw_y[i];
  const int col0 = blockIdx.x * kCB;
  for (int i = threadIdx.x; i < ny * kCB; i += blockDim.x) {
    const int ky = i / kCB, c = i - ky * kCB;
    const int col = col0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (col < ncols) v = T[((size_t)z * ny + ky) * ncols + col];
    a[c * bs + ky] = cscale(v, sgn(ky + ny / 2) * g.inv_sqrt_ny);
  }
  __syncthreads();
  float2* res = fft_batch<+1>(a, b, kCB, bs, g.fy, tw, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < ny * kCB; i += blockDim.x) {
    const int y = i / kCB, c = i - y * kCB;
    const int col = col0 + c;
    if (col < ncols) H[((size_t)z * ny + y) * ncols + col] = cscale(res[c * bs + y], sgn(y));
  }
}

// mode 0: forward gather (T -> Sc); mode 1: adjoint scatter (Sc -> T);
// mode 2: normal projection in place on T with ||.||^2 into *qq.
__global__ void __launch_bounds__(kK2Threads) k2_z_3d(Geo g, float2* __restrict__ T, float2* __restrict__ Sc,
                                                      int ncols, int mode, double* partials,
                                                      unsigned* counter, double* qq) {
  extern __shared__ float2 smem[];
  __shared__ double red[32];
  const int ny = g.ny, nz = g.nz, bs = nz + 1, ky = blockIdx.y;
  float2* a = smem;
  float2* b = smem + kCB * bs;
  float2* tw = smem + 2 * kCB * bs;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = g.tw_z[i];
  const int col0 = blockIdx.x * kCB;
  if (mode == 1) {
    for (int i = threadIdx.x; i < kCB * bs; i += blockDim.x) a[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < nz * kCB; i += blockDim.x) {
      const int kz = i / kCB, c = i - kz * kCB;
      const int col = col0 + c;
      const int l = g.line_of[kz * ny + ky];
      if (l >= 0 && col < ncols)
        a[c * bs + kz] = cscale(Sc[(size_t)l * ncols + col], sgn(kz + nz / 2) * g.inv_sqrt_nz);
    }
    __syncthreads();
    float2* res = fft_batch<+1>(a, b, kCB, bs, g.fz, tw, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < nz * kCB; i += blockDim.x) {
      const int z = i / kCB, c = i - z * kCB;
      const int col = col0 + c;
      if (col < ncols) T[((size_t)z * ny + ky) * ncols + col] = cscale(res[c * bs + z], sgn(z));
    }
    return;
  }
  for (int i = threadIdx.x; i < nz * kCB; i += blockDim.x) {
    const int z = i / kCB, c = i - z * kCB;
    const int col = col0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (col < ncols) v = T[((size_t)z * ny + ky) * ncols + col];
    a[c * bs + z] = cscale(v, sgn(z));
  }
  __syncthreads();
  float2* res = fft_batch<-1>(a, b, kCB, bs, g.fz, tw, threadIdx.x, blockDim.x);
  if (mode == 0) {
    for (int i = threadIdx.x; i < nz * kCB; i += blockDim.x) {
      const int kz = i / kCB, c = i - kz * kCB;
      const int col = col0 + c;
      const int l = g.line_of[kz * ny + ky];
      if (l >= 0 && col < ncols)
        Sc[(size_t)l * ncols + col] = cscale(res[c * bs + kz], sgn(kz + nz / 2) * g.inv_sqrt_nz);
    }
    return;
  }
  float2* oth = (res == a) ? b : a;
  const float inv_nz = 1.0f / (float)nz;
  double part = 0.0;
  for (int i = threadIdx.x; i < nz * kCB; i += blockDim.x) {
    const int c = i / nz, kz = i - c * nz;
    float2 v = res[c * bs + kz];
    if (g.line_of[kz * ny + ky] >= 0 && col0 + c < ncols) {
      part += ((double)v.x * v.x + (double)v.y * v.y) * inv_nz;
      v = cscale(v, inv_nz);
    } else {
      v = make_float2(0.f, 0.f);
    }
    res[c * bs + kz] = v;
  }
  __syncthreads();
  float2* res2 = fft_batch<+1>(res, oth, kCB, bs, g.fz, tw, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < nz * kCB; i += blockDim.x) {
    const int z = i / kCB, c = i - z * kCB;
    const int col = col0 + c;
    if (col < ncols) T[((size_t)z * ny + ky) * ncols + col] = cscale(res2[c * bs + z], sgn(z));
  }
  if (qq) grid_sum_finalize(part, partials, counter, qq, red);
}

// ------------------------------------------------------------------ launchers --
static size_t k2_smem(int n) { return sizeof(float2) * (size_t)(2 * kCB * (n + 1) + n); }

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

static void set_k2_attr(const void* f, size_t sm) {
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

cudaError_t launch_pe_fwd(const Geo& g, const float2* Hpart, int nchunk, int ncols, float2* T, float2* Sc,
                          cudaStream_t st) {
  const int nb = (ncols + kCB - 1) / kCB;
  if (!g.dim3d) {
    const size_t sm = k2_smem(g.ny);
    set_k2_attr((const void*)k2_fwd_2d, sm);
    note_launches(1); k2_fwd_2d<<<nb, kK2Threads, sm, st>>>(g, Hpart, nchunk, ncols, Sc);
    return cudaGetLastError();
  }
  size_t sm = k2_smem(g.ny);
  set_k2_attr((const void*)k2_y_fwd3d, sm);
  note_launches(1); k2_y_fwd3d<<<dim3(nb, g.nz), kK2Threads, sm, st>>>(g, Hpart, nchunk, ncols, T);
  sm = k2_smem(g.nz);
  set_k2_attr((const void*)k2_z_3d, sm);
  note_launches(1); k2_z_3d<<<dim3(nb, g.ny), kK2Threads, sm, st>>>(g, T, Sc, ncols, 0, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pe_adj(const Geo& g, const float2* Sc, int ncols, float2* T, float2* H, cudaStream_t st) {
  const int nb = (ncols + kCB - 1) / kCB;
  if (!g.dim3d) {
    const size_t sm = k2_smem(g.ny);
    set_k2_attr((const void*)k2_adj_2d, sm);
    note_launches(1); k2_adj_2d<<<nb, kK2Threads, sm, st>>>(g, Sc, ncols, H);
    return cudaGetLastError();
  }
  size_t sm = k2_smem(g.nz);
  set_k2_attr((const void*)k2_z_3d, sm);
  note_launches(1); k2_z_3d<<<dim3(nb, g.ny), kK2Threads, sm, st>>>(g, T, (float2*)Sc, ncols, 1, nullptr, nullptr, nullptr);
  sm = k2_smem(g.ny);
  set_k2_attr((const void*)k2_y_adj3d, sm);
  note_launches(1); k2_y_adj3d<<<dim3(nb, g.nz), kK2Threads, sm, st>>>(g, T, ncols, H);
  return cudaGetLastError();
}

int pe_normal_blocks(const Geo& g, int ncols) {
  const int nb = (ncols + kCB - 1) / kCB;
  return g.dim3d ? nb * g.ny : nb;
}

cudaError_t launch_pe_normal(const Geo& g, const float2* Hpart, int nchunk, int ncols, float2* T, float2* H2,
                             double* partials, unsigned* counter, double* qq, cudaStream_t st) {
  const int nb = (ncols + kCB - 1) / kCB;
  if (!g.dim3d) {
    const size_t sm = k2_smem(g.ny);
    set_k2_attr((const void*)k2_normal_2d, sm);
    note_launches(1); k2_normal_2d<<<nb, kK2Threads, sm, st>>>(g, Hpart, nchunk, ncols, H2, partials, counter, qq);
    return cudaGetLastError();
  }
  size_t sm = k2_smem(g.ny);
  set_k2_attr((const void*)k2_y_fwd3d, sm);
  note_launches(1); k2_y_fwd3d<<<dim3(nb, g.nz), kK2Threads, sm, st>>>(g, Hpart, nchunk, ncols, T);
  sm = k2_smem(g.nz);
  set_k2_attr((const void*)k2_z_3d, sm);
  note_launches(1); k2_z_3d<<<dim3(nb, g.ny), kK2Threads, sm, st>>>(g, T, nullptr, ncols, 2, partials, counter, qq);
  sm = k2_smem(g.ny);
  set_k2_attr((const void*)k2_y_adj3d, sm);
  note_launches(1); k2_y_adj3d<<<dim3(nb, g.nz), kK2Threads, sm, st>>>(g, T, ncols, H2);
  return cudaGetLastError();
}

}  // namespace gpjc
