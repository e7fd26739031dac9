// Uncompressed readout stage, C then Psi F_ro (Eq. 1-4): the spectra
// V[row][n][t] of every coil, FP32 or 16-bit.  Used by the acquisition model
// (gpjc_simulate and its adjoint) and as the first half of the 16-bit
// tensor-core operators, whose A_g products run in k_tc.cu.
//
// One block per (phase-encode row, coil chunk).  The zero-padded N_tx-point
// readout DFT of an N_x-point row is computed as os twiddled N_x-point FFTs
// (t = os m + s), followed by the wave / centring factor post(t, y, z).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <type_traits>

#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kK1Threads = 256;

// -------------------------------------------------------------------------
// Uncompressed readout stage (the acquisition model E, and the first half of
// the BF16 operator): V[row][n][t] = Psi F_ro (c_n x) for each coil.
template <typename VT>
__device__ __forceinline__ void store_v(VT* p, float2 v);
template <>
__device__ __forceinline__ void store_v<float2>(float2* p, float2 v) { *p = v; }
template <>
__device__ __forceinline__ void store_v<__nv_bfloat162>(__nv_bfloat162* p, float2 v) {
  *p = __floats2bfloat162_rn(v.x, v.y);
}
template <>
__device__ __forceinline__ void store_v<__half2>(__half2* p, float2 v) {
  *p = __floats2half2_rn(v.x, v.y);
}
template <typename VT>
__device__ __forceinline__ float2 load_v(const VT* p);
template <>
__device__ __forceinline__ float2 load_v<__half2>(const __half2* p) {
  return __half22float2(*p);
}
template <>
__device__ __forceinline__ float2 load_v<float2>(const float2* p) { return *p; }
template <>
__device__ __forceinline__ float2 load_v<__nv_bfloat162>(const __nv_bfloat162* p) {
  return __bfloat1622float2(*p);
}

// smem: two padded ntx buffers + twiddles; post / pre are read from their
// global tables (L2 / L1 resident) in coalesced order
static size_t sim_smem(const Geo& g) { return sizeof(float2) * (size_t)(2 * spad_size(g.ntx) + g.nx); }

__device__ __forceinline__ float2 post_of(const Geo& g, int t, int row) {
  const int y = row % g.ny, z = row / g.ny;
  const float2 py = __ldg(g.post_y + (size_t)y * g.ntx + t);
  if (g.nz == 1) return py;
  return cmul(py, __ldg(g.post_z + (size_t)z * g.ntx + t));
}

template <typename VT>
__global__ void __launch_bounds__(kK1Threads) k1_sim_fwd(Geo g, const float2* __restrict__ x,
                                                         const float2* __restrict__ coil,
                                                         VT* __restrict__ V, int cpc, int row0) {
  extern __shared__ float2 smem[];
  float2* A = smem;
  float2* B = A + spad_size(g.ntx);
  float2* tw = B + spad_size(g.ntx);
  const int row = row0 + blockIdx.x, chunk = blockIdx.y;
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * g.nx;
  const int nx = g.nx, os = g.os;
  const float2* xrow = x + (size_t)row * nx;
  const int n0 = chunk * cpc;
  const int n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; ++n) {
    const float2* crow = coil + n * L + (size_t)row * nx;
    for (int i = threadIdx.x; i < g.ntx; i += blockDim.x) {
      const int xx = i % nx;
      A[spad(i)] = cmul(cmul(__ldg(crow + xx), __ldg(xrow + xx)), __ldg(g.pre + i));
    }
    __syncthreads();
    const float2* R = fft_batch<-1, true>(A, B, os, nx, g.fx, tw, threadIdx.x, blockDim.x);
    VT* out = V + ((size_t)row * g.nc + n) * g.ntx;
    for (int t = threadIdx.x; t < g.ntx; t += blockDim.x) {
      const int m = t / os, s = t - m * os;
      store_v<VT>(out + t, cmul(R[spad(s * nx + m)], post_of(g, t, row)));
    }
    __syncthreads();
  }
}

template <typename VT, int MAXX>
__global__ void __launch_bounds__(kK1Threads) k1_sim_adj(Geo g, const VT* __restrict__ V,
                                                         const float2* __restrict__ coil,
                                                         float2* __restrict__ xpart, int cpc, int row0) {
  extern __shared__ float2 smem[];
  float2* A = smem;
  float2* B = A + spad_size(g.ntx);
  float2* tw = B + spad_size(g.ntx);
  const int row = row0 + blockIdx.x, chunk = blockIdx.y;
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * g.nx;
  const int nx = g.nx, os = g.os;
  float2 xacc[MAXX];
#pragma unroll
  for (int j = 0; j < MAXX; ++j) xacc[j] = make_float2(0.f, 0.f);
  const int n0 = chunk * cpc;
  const int n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; ++n) {
    const VT* vin = V + ((size_t)row * g.nc + n) * g.ntx;
    for (int t = threadIdx.x; t < g.ntx; t += blockDim.x) {
      const int m = t / os, s = t - m * os;
      A[spad(s * nx + m)] = cmulc(post_of(g, t, row), load_v<VT>(vin + t));
    }
    __syncthreads();
    const float2* R = fft_batch<+1, true>(A, B, os, nx, g.fx, tw, threadIdx.x, blockDim.x);
    const float2* crow = coil + n * L + (size_t)row * nx;
#pragma unroll
    for (int j = 0; j < MAXX; ++j) {
      const int xx = threadIdx.x + j * kK1Threads;
      if (xx < nx) {
        float2 u = make_float2(0.f, 0.f);
        for (int s = 0; s < os; ++s) cfmac(u, __ldg(g.pre + s * nx + xx), R[spad(s * nx + xx)]);
        cfmac(xacc[j], __ldg(crow + xx), u);
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

// Two-pass variants of the two kernels above (readout lengths with a
// two-pass FFT plan, g.fx.n1 > 0).  NB coils go through one FFT call, so
// that the os NB transforms give every thread of the block a column in both
// passes; the forward kernel forms u = c_n x once per pixel and applies the
// pre-twiddle while the first pass loads, the adjoint applies it in the coil
// sum.  The spectra sit in shared memory in natural order t = os m + s,
// padded one slot in nine (conflict-free for the stride-os reads of a pass).
constexpr int kSimMaxNB = 2;
template <int NB>
static size_t sim2_smem(const Geo& g) {
  return sizeof(float2) * (size_t)(spad_size(NB * g.ntx) + NB * g.ntx + NB * g.nx + g.nx);
}

template <typename VT, int NB>
__global__ void __launch_bounds__(kK1Threads) k1_sim_fwd2(Geo g, const float2* __restrict__ x,
                                                          const float2* __restrict__ coil,
                                                          VT* __restrict__ V, int cpc, int row0) {
  static_assert(NB >= 1 && NB <= kSimMaxNB, "one or two coils per FFT call");
  extern __shared__ float2 smem[];
  const int nx = g.nx, os = g.os, ntx = g.ntx;
  float2* O = smem;                     // spectra of the NB coils, padded, natural order
  float2* B = O + spad_size(NB * ntx);  // FFT scratch
  float2* u = B + NB * ntx;             // c_n x of the NB coils
  float2* tw = u + NB * nx;
  const int row = row0 + blockIdx.x, chunk = blockIdx.y;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * nx;
  const float2* xrow = x + (size_t)row * nx;
  const int n0 = chunk * cpc, n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; n += NB) {
    const int nb = min(NB, n1 - n);
    for (int i = threadIdx.x; i < nb * nx; i += blockDim.x) {
      const int j = i >= nx ? 1 : 0, xx = i - j * nx;
      u[i] = cmul(__ldg(coil + (n + j) * L + (size_t)row * nx + xx), __ldg(xrow + xx));
    }
    __syncthreads();
    auto ld = [&](int f, int xx) {
      const int j = (NB > 1 && f >= os) ? 1 : 0, s = f - j * os;
      return cmul(u[j * nx + xx], __ldg(g.pre + s * nx + xx));
    };
    auto st = [&](int f, int m, float2 v) {
      const int j = (NB > 1 && f >= os) ? 1 : 0, s = f - j * os;
      O[spad(j * ntx + m * os + s)] = v;
    };
    fft2p_cb_dispatch<-1>(g.fx.n1, g.fx.n2, ld, st, B, nb * os, tw, threadIdx.x, blockDim.x);
    VT* out = V + ((size_t)row * g.nc + n) * ntx;  // coils n .. n + nb - 1 are contiguous
    for (int i = threadIdx.x; i < nb * ntx; i += blockDim.x) {
      const int t = i >= ntx ? i - ntx : i;
      store_v<VT>(out + i, cmul(O[spad(i)], post_of(g, t, row)));
    }
    // u and O are rewritten only after the next pair's first barrier
  }
}

template <typename VT, int NB, int MAXX>
__global__ void __launch_bounds__(kK1Threads) k1_sim_adj2(Geo g, const VT* __restrict__ V,
                                                          const float2* __restrict__ coil,
                                                          float2* __restrict__ xpart, int cpc, int row0) {
  static_assert(NB >= 1 && NB <= kSimMaxNB, "one or two coils per FFT call");
  extern __shared__ float2 smem[];
  const int nx = g.nx, os = g.os, ntx = g.ntx;
  float2* O = smem;                     // staged spectra (padded), then the FFT outputs (plain)
  float2* B = O + spad_size(NB * ntx);  // FFT scratch
  float2* tw = B + NB * ntx;
  const int row = row0 + blockIdx.x, chunk = blockIdx.y;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * nx;
  float2 xacc[MAXX];
#pragma unroll
  for (int j = 0; j < MAXX; ++j) xacc[j] = make_float2(0.f, 0.f);
  const int n0 = chunk * cpc, n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; n += NB) {
    const int nb = min(NB, n1 - n);
    const VT* vin = V + ((size_t)row * g.nc + n) * ntx;
    // loads first, four elements per thread at a time, so their latencies overlap
    for (int i0 = threadIdx.x; i0 < nb * ntx; i0 += 4 * blockDim.x) {
      float2 v[4], p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < nb * ntx) {
          v[u] = load_v<VT>(vin + i);
          p[u] = post_of(g, i >= ntx ? i - ntx : i, row);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < nb * ntx) O[spad(i)] = cmulc(p[u], v[u]);
      }
    }
    __syncthreads();
    auto ld = [&](int f, int m) {
      const int j = (NB > 1 && f >= os) ? 1 : 0, s = f - j * os;
      return O[spad(j * ntx + m * os + s)];
    };
    // the staged spectra are consumed by the first pass; transform f's
    // output goes to O[f nx ...]
    auto st = [&](int f, int xx, float2 v) { O[f * nx + xx] = v; };
    fft2p_cb_dispatch<+1>(g.fx.n1, g.fx.n2, ld, st, B, nb * os, tw, threadIdx.x, blockDim.x);
#pragma unroll
    for (int j = 0; j < MAXX; ++j) {
      const int xx = threadIdx.x + j * kK1Threads;
      if (xx < nx) {
        float2 cv[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c)
          cv[c] = c < nb ? __ldg(coil + (n + c) * L + (size_t)row * nx + xx) : make_float2(0.f, 0.f);
        float2 uu[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) uu[c] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int s = 0; s < os; ++s) {
          const float2 pr = __ldg(g.pre + s * nx + xx);  // shared by the NB coils
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c < nb) cfmac(uu[c], pr, O[c * ntx + s * nx + xx]);
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < nb) cfmac(xacc[j], cv[c], uu[c]);
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

// ------------------------------------------------------------------ host side --
// (left out when the kernels above are compiled for a host emulation)
#ifndef GPJC_DEVICE_SOURCE_ONLY
constexpr size_t kSimSmemMax = 200 * 1024;

// GPJC_SIM_LEGACY=1 keeps the one-coil kernels on two-pass lengths too (on the
// 256 x 256, 32-coil BF16 FISTA step the two-coil forward saved 2 ms of 43,
// the two-coil adjoint 0.25 ms of 39)
static bool sim_two_pass(const Geo& g) {
  static int legacy = -1;
  if (legacy < 0) {
    const char* e = getenv("GPJC_SIM_LEGACY");
    legacy = (e && e[0] == '1') ? 1 : 0;
  }
  return !legacy && g.fx.n1 > 0 && sim2_smem<2>(g) <= kSimSmemMax;
}

template <typename VT, int NB>
static cudaError_t launch_sim_fwd2(const Geo& g, const float2* x, const float2* coil, VT* V, int cpc, dim3 grid,
                                   int row0, cudaStream_t st) {
  const size_t sm = sim2_smem<NB>(g);
  cudaFuncSetAttribute(k1_sim_fwd2<VT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k1_sim_fwd2<VT, NB><<<grid, kK1Threads, sm, st>>>(g, x, coil, V, cpc, row0);
  return cudaGetLastError();
}

template <typename VT, int NB, int MAXX>
static cudaError_t launch_sim_adj2(const Geo& g, const VT* V, const float2* coil, float2* xpart, int cpc, dim3 grid,
                                   int row0, cudaStream_t st) {
  const size_t sm = sim2_smem<NB>(g) - sizeof(float2) * (size_t)(NB * g.nx);  // no u buffer
  cudaFuncSetAttribute(k1_sim_adj2<VT, NB, MAXX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k1_sim_adj2<VT, NB, MAXX><<<grid, kK1Threads, sm, st>>>(g, V, coil, xpart, cpc, row0);
  return cudaGetLastError();
}

// rows [row0, row0 + nrows) of the forward readout
template <typename VT>
static cudaError_t launch_sim_fwd_t(const Geo& g, const float2* x, const float2* coil, VT* V, int nchunk,
                                    int row0, int nrows, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  dim3 grid(nrows, nchunk);
  if (sim_two_pass(g)) return launch_sim_fwd2<VT, 2>(g, x, coil, V, cpc, grid, row0, st);
  const size_t sm = sim_smem(g);
  cudaFuncSetAttribute(k1_sim_fwd<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k1_sim_fwd<VT><<<grid, kK1Threads, sm, st>>>(g, x, coil, V, cpc, row0);
  return cudaGetLastError();
}

// rows [row0, row0 + nrows) of the adjoint readout
template <typename VT>
static cudaError_t launch_sim_adj_t(const Geo& g, const VT* V, const float2* coil, float2* xpart, int nchunk,
                                    int row0, int nrows, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  dim3 grid(nrows, nchunk);
  // (FP32 spectra only: the adjoint of the 16-bit operators expands into FP32)
  if constexpr (std::is_same<VT, float2>::value)
    if (sim_two_pass(g))
      return g.nx <= kK1Threads ? launch_sim_adj2<VT, 2, 1>(g, V, coil, xpart, cpc, grid, row0, st)
                                : launch_sim_adj2<VT, 2, 2>(g, V, coil, xpart, cpc, grid, row0, st);
  const size_t sm = sim_smem(g);
  if (g.nx <= kK1Threads) {
    cudaFuncSetAttribute(k1_sim_adj<VT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launches(1); k1_sim_adj<VT, 1><<<grid, kK1Threads, sm, st>>>(g, V, coil, xpart, cpc, row0);
  } else {
    cudaFuncSetAttribute(k1_sim_adj<VT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launches(1); k1_sim_adj<VT, 2><<<grid, kK1Threads, sm, st>>>(g, V, coil, xpart, cpc, row0);
  }
  return cudaGetLastError();
}

cudaError_t launch_sim_fwd(const Geo& g, const float2* x, const float2* coil, float2* V, int nchunk,
                           cudaStream_t st) {
  return launch_sim_fwd_t<float2>(g, x, coil, V, nchunk, 0, g.rows, st);
}
cudaError_t launch_sim_fwd_rows(const Geo& g, const float2* x, const float2* coil, float2* V, int nchunk, int row0,
                                int nrows, cudaStream_t st) {
  return launch_sim_fwd_t<float2>(g, x, coil, V, nchunk, row0, nrows, st);
}
cudaError_t launch_sim_fwd_f16(const Geo& g, const float2* x, const float2* coil, void* V, int nchunk,
                               int row0, int nrows, cudaStream_t st) {
  return launch_sim_fwd_t<__half2>(g, x, coil, (__half2*)V, nchunk, row0, nrows, st);
}
cudaError_t launch_sim_adj_f16(const Geo& g, const void* V, const float2* coil, float2* xpart, int nchunk,
                               cudaStream_t st) {
  return launch_sim_adj_t<__half2>(g, (const __half2*)V, coil, xpart, nchunk, 0, g.rows, st);
}
cudaError_t launch_sim_adj(const Geo& g, const float2* V, const float2* coil, float2* xpart, int nchunk,
                           cudaStream_t st) {
  return launch_sim_adj_t<float2>(g, V, coil, xpart, nchunk, 0, g.rows, st);
}
cudaError_t launch_sim_adj_rows(const Geo& g, const float2* V, const float2* coil, float2* xpart, int nchunk,
                                int row0, int nrows, cudaStream_t st) {
  return launch_sim_adj_t<float2>(g, V, coil, xpart, nchunk, row0, nrows, st);
}

#endif  // GPJC_DEVICE_SOURCE_ONLY

}  // namespace gpjc
