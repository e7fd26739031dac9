// Phase-encode stage of the matrix-free encoding operators (Eq. 4, 15): one
// block per 8-column slab of the hybrid matrix H[row][col]; FFT along y
// (and z in 3D), gather / scatter of the sampled lines, and for E_c^H E_c
// the fused mask projection with the squared norm ||E_c p||^2 accumulated
// for CG.
#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kK2Threads = 256;
constexpr int kCB = 8;  // columns per phase-encode block (8: 512 blocks on 2d256, 13 us per launch; 16: 256 blocks, 16 us)

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
