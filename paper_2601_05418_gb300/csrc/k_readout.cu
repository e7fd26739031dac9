// Readout stage of E_c and E_c^H, FP32, register-tiled (Eq. 13-15).
//
// A block owns RB phase-encode rows and a chunk of coils.  Per coil, each
// row's zero-padded readout DFT is computed as os pre-twiddled N_x-point
// Stockham FFTs in (bank-padded) shared memory and multiplied by the wave /
// centring factor post(t, y, z); the spectra of the RB rows stay in shared
// memory while the group compression runs as many small GEMMs
//   H[(row, p), k] += sum_tau A_g[k][n w + tau] U_row[p w + tau],
// one register tile of 4 kept components x 4 patch columns per thread
// (16 complex accumulators, 8 loads per 16 complex multiply-adds).  The
// adjoint applies A_g^H with tiles of 4 readout samples x 4 columns, then
// inverse FFTs each row and accumulates conj(c_n) times the result.
//
// The tiles (group, first kept component / first sample, up to 4 columns)
// are listed on the host per geometry and RB (plan tables), so any patch ->
// group map and any per-group keep are handled by the same kernels.
#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kRThreads = 256;

// logical row stride of the spectra in shared memory (multiple of 8, so a
// row's padded sub-buffer starts at spad(r * stride))
__host__ __device__ inline int u_stride(int ntx) { return (ntx + 7) & ~7; }

size_t readout_fwd_smem(const Geo& g, int rb) {
  const int st = u_stride(g.ntx);
  return sizeof(float2) * (size_t)(spad_size(rb * st) + 2 * spad_size(g.ntx) + g.nx);
}
size_t readout_adj_smem(const Geo& g, int rb) {
  const int st = u_stride(g.ntx);
  return sizeof(float2) * (size_t)(spad_size(rb * st) + spad_size(g.ntx) + g.nx);
}

__device__ __forceinline__ float2 post_at(const Geo& g, int t, int row) {
  const int y = row % g.ny, z = row / g.ny;
  const float2 py = g.post_y[(size_t)y * g.ntx + t];
  if (g.nz == 1) return py;
  return cmul(py, g.post_z[(size_t)z * g.ntx + t]);
}

// ------------------------------------------------------------------ forward --
template <int MAXT>
__global__ void __launch_bounds__(kRThreads) k1f_tiled(Geo g, RTiles tl, const float2* __restrict__ x,
                                                       const float2* __restrict__ coil,
                                                       const float2* __restrict__ AT, float2* __restrict__ Hpart,
                                                       int cpc) {
  extern __shared__ float2 rsm[];
  const int rb = tl.rb, st = u_stride(g.ntx);
  float2* U = rsm;
  float2* A = U + spad_size(rb * st);
  float2* B = A + spad_size(g.ntx);
  float2* tw = B + spad_size(g.ntx);
  const int row0 = blockIdx.x * rb, chunk = blockIdx.y;
  const int nrows = min(rb, g.rows - row0);
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * g.nx;
  const int nx = g.nx, os = g.os, w = g.w;

  float2 acc[MAXT][4][4];
  int4 hdr[MAXT];
  int uoff[MAXT][4];
#pragma unroll
  for (int m = 0; m < MAXT; ++m) {
    const int tile = threadIdx.x + m * kRThreads;
    hdr[m] = tile < tl.nt ? tl.hdr[tile] : make_int4(0, 1, 0, 0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int4 cc = tile < tl.nt ? tl.cols[tile * 4 + c] : make_int4(-1, -1, 0, 0);
      // columns of rows past the end of the grid are dropped
      uoff[m][c] = (cc.x >= 0 && cc.x / st < nrows) ? cc.x : -1;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[m][c][k] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const int n0 = chunk * cpc, n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; ++n) {
    for (int r = 0; r < nrows; ++r) {
      const int row = row0 + r;
      const float2* crow = coil + n * L + (size_t)row * nx;
      const float2* xrow = x + (size_t)row * nx;
      for (int i = threadIdx.x; i < g.ntx; i += blockDim.x) {
        const int xx = i % nx;
        A[spad(i)] = cmul(cmul(__ldg(crow + xx), __ldg(xrow + xx)), __ldg(g.pre + i));
      }
      __syncthreads();
      float2* R = fft_batch<-1, true>(A, B, os, nx, g.fx, tw, threadIdx.x, blockDim.x);
      float2* Ur = U + spad(r * st);
      for (int i = threadIdx.x; i < g.ntx; i += blockDim.x) {
        const int s = i / nx, m = i - s * nx;
        const int t = m * os + s;
        Ur[spad(t)] = cmul(R[spad(i)], post_at(g, t, row));
      }
      __syncthreads();
    }
    const int nw = n * w;
#pragma unroll
    for (int m = 0; m < MAXT; ++m) {
      const int4 h = hdr[m];  // (aoff_g + k0, keep_g, kcnt, unused)
      if (h.z == 0) continue;
      const float2* Ap = AT + h.x + (size_t)nw * h.y;
      for (int tau = 0; tau < w; ++tau) {
        float2 a[4], u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = k < h.z ? __ldg(Ap + k) : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) u[c] = uoff[m][c] >= 0 ? U[spad(uoff[m][c] + tau)] : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) cfma(acc[m][c][k], a[k], u[c]);
        Ap += h.y;
      }
    }
    __syncthreads();
  }
  float2* out = Hpart + ((size_t)chunk * g.rows + row0) * g.ntxc;
#pragma unroll
  for (int m = 0; m < MAXT; ++m) {
    const int tile = threadIdx.x + m * kRThreads;
    if (tile >= tl.nt) continue;
    const int kc = hdr[m].z;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (uoff[m][c] < 0) continue;
      const int o = tl.cols[tile * 4 + c].y;  // r * ntxc + off_p + k0
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < kc) out[o + k] = acc[m][c][k];
    }
  }
}

// ------------------------------------------------------------------ adjoint --
template <int MAXX>
__global__ void __launch_bounds__(kRThreads) k1a_tiled(Geo g, RTiles tl, const float2* __restrict__ H2,
                                                       const float2* __restrict__ coil,
                                                       const float2* __restrict__ Arow, float2* __restrict__ xpart,
                                                       int cpc) {
  extern __shared__ float2 rsm[];
  const int rb = tl.rb, st = u_stride(g.ntx);
  float2* U = rsm;
  float2* B = U + spad_size(rb * st);
  float2* tw = B + spad_size(g.ntx);
  const int row0 = blockIdx.x * rb, chunk = blockIdx.y;
  const int nrows = min(rb, g.rows - row0);
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * g.nx;
  const int nx = g.nx, os = g.os, w = g.w, ns = g.ns;

  float2 xacc[MAXX];
#pragma unroll
  for (int j = 0; j < MAXX; ++j) xacc[j] = make_float2(0.f, 0.f);
  __syncthreads();
  const int n0 = chunk * cpc, n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; ++n) {
    // A^H on every tile: U_r[t] = sum_k conj(A_g[k][n w + tau]) H2[row][off_p + k];
    // the tile descriptors are re-read (L1) to keep registers for the sums
    for (int tile = threadIdx.x; tile < tl.nt; tile += kRThreads) {
      const int4 h = tl.hdr[tile];  // (aoff_g + tau0, keep_g, tcnt, unused)
      int cr[4];
      const float2* hp[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int4 cc = tl.cols[tile * 4 + c];  // (r, off_p, p w + tau0, 0)
        cr[c] = (cc.x >= 0 && cc.x < nrows) ? cc.x : -1;
        hp[c] = cr[c] >= 0 ? H2 + (size_t)(row0 + cc.x) * g.ntxc + cc.y : H2;
      }
      float2 acc[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[c][k] = make_float2(0.f, 0.f);
      const float2* Ap = Arow + h.x + n * w;
      for (int k = 0; k < h.y; ++k) {
        float2 a[4], hv[4];
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) a[tt] = tt < h.z ? __ldg(Ap + tt) : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) hv[c] = cr[c] >= 0 ? __ldg(hp[c] + k) : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int tt = 0; tt < 4; ++tt) cfmac(acc[c][tt], a[tt], hv[c]);
        Ap += ns;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (cr[c] < 0) continue;
        float2* Ur = U + spad(cr[c] * st);
        const int t0 = tl.cols[tile * 4 + c].z;
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
          if (tt >= h.z) continue;
          const int t = t0 + tt;
          const int mm = t / os, s = t - mm * os;
          Ur[spad(s * nx + mm)] = cmulc(post_at(g, t, row0 + cr[c]), acc[c][tt]);
        }
      }
    }
    __syncthreads();
    for (int r = 0; r < nrows; ++r) {
      float2* Ur = U + spad(r * st);
      float2* R = fft_batch<+1, true>(Ur, B, os, nx, g.fx, tw, threadIdx.x, blockDim.x);
      const float2* crow = coil + n * L + (size_t)(row0 + r) * nx;
      // thread-owned output slots (r', x) = slot / nx, slot % nx
#pragma unroll
      for (int j = 0; j < MAXX; ++j) {
        const int slot = threadIdx.x + j * kRThreads;
        if (slot < nrows * nx && slot / nx == r) {
          const int xx = slot - r * nx;
          float2 u = make_float2(0.f, 0.f);
          for (int s = 0; s < os; ++s) cfmac(u, __ldg(g.pre + s * nx + xx), R[spad(s * nx + xx)]);
          cfmac(xacc[j], __ldg(crow + xx), u);
        }
      }
      __syncthreads();
    }
  }
  float2* out = xpart + ((size_t)chunk * g.rows + row0) * nx;
#pragma unroll
  for (int j = 0; j < MAXX; ++j) {
    const int slot = threadIdx.x + j * kRThreads;
    if (slot < nrows * nx) out[slot] = xacc[j];
  }
}

}  // namespace gpjc

namespace gpjc {

// ------------------------------------------------------------------ host side --
static int ceil_div(int a, int b) { return (a + b - 1) / b; }

void build_readout_tiles(const ReadoutGeomHost& h, int rb, bool adjoint, std::vector<int4>* hdr,
                         std::vector<int4>* cols) {
  const int st = u_stride(h.ntx);
  std::vector<std::vector<int>> occ(h.G);
  for (int p = 0; p < (int)h.pg.size(); ++p) occ[h.pg[p]].push_back(p);
  hdr->clear();
  cols->clear();
  for (int g = 0; g < h.G; ++g) {
    const int oc = (int)occ[g].size();
    const int ncol = rb * oc;
    const int inner = adjoint ? h.w : h.keep[g];  // samples (adjoint) or kept components (forward)
    for (int i0 = 0; i0 < inner; i0 += 4) {
      for (int c0 = 0; c0 < ncol; c0 += 4) {
        hdr->push_back(make_int4(h.aoff[g] + i0, h.keep[g], std::min(4, inner - i0), 0));
        for (int c = 0; c < 4; ++c) {
          const int cc = c0 + c;
          if (cc >= ncol) {
            cols->push_back(make_int4(-1, -1, 0, 0));
            continue;
          }
          const int r = cc / oc, p = occ[g][cc % oc];
          if (adjoint)
            cols->push_back(make_int4(r, h.poff[p], p * h.w + i0, 0));
          else
            cols->push_back(make_int4(r * st + p * h.w, r * h.ntxc + h.poff[p] + i0, 0, 0));
        }
      }
    }
  }
}

int readout_tile_count(const ReadoutGeomHost& h, int rb, bool adjoint) {
  std::vector<std::vector<int>> occ(h.G);
  for (int p = 0; p < (int)h.pg.size(); ++p) occ[h.pg[p]].push_back(p);
  int n = 0;
  for (int g = 0; g < h.G; ++g)
    n += ceil_div(adjoint ? h.w : h.keep[g], 4) * ceil_div(rb * (int)occ[g].size(), 4);
  return n;
}

template <int MAXT>
static cudaError_t launch_f(const Geo& g, const RTiles& tl, const float2* x, const float2* coil, const float2* AT,
                            float2* Hpart, int nchunk, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  const size_t sm = readout_fwd_smem(g, tl.rb);
  static int attr = 0;
  if ((int)sm > attr) {
    cudaFuncSetAttribute(k1f_tiled<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k1f_tiled<MAXT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = (int)sm;
  }
  dim3 grid((g.rows + tl.rb - 1) / tl.rb, nchunk);
  note_launches(1); k1f_tiled<MAXT><<<grid, kRThreads, sm, st>>>(g, tl, x, coil, AT, Hpart, cpc);
  return cudaGetLastError();
}

cudaError_t launch_k1f_tiled(const Geo& g, const RTiles& tl, const float2* x, const float2* coil,
                             const float2* AT, float2* Hpart, int nchunk, cudaStream_t st) {
  const int maxt = ceil_div(tl.nt, kRThreads);
  if (maxt <= 1) return launch_f<1>(g, tl, x, coil, AT, Hpart, nchunk, st);
  if (maxt <= 2) return launch_f<2>(g, tl, x, coil, AT, Hpart, nchunk, st);
  if (maxt <= 3) return launch_f<3>(g, tl, x, coil, AT, Hpart, nchunk, st);
  return cudaErrorInvalidValue;
}

template <int MAXX>
static cudaError_t launch_a(const Geo& g, const RTiles& tl, const float2* H2, const float2* coil,
                            const float2* A, float2* xpart, int nchunk, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  const size_t sm = readout_adj_smem(g, tl.rb);
  static int attr = 0;
  if ((int)sm > attr) {
    cudaFuncSetAttribute(k1a_tiled<MAXX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k1a_tiled<MAXX>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = (int)sm;
  }
  dim3 grid((g.rows + tl.rb - 1) / tl.rb, nchunk);
  note_launches(1); k1a_tiled<MAXX><<<grid, kRThreads, sm, st>>>(g, tl, H2, coil, A, xpart, cpc);
  return cudaGetLastError();
}

cudaError_t launch_k1a_tiled(const Geo& g, const RTiles& tl, const float2* H2, const float2* coil,
                             const float2* A, float2* xpart, int nchunk, cudaStream_t st) {
  const int mx = ceil_div(tl.rb * g.nx, kRThreads);
  if (mx <= 1) return launch_a<1>(g, tl, H2, coil, A, xpart, nchunk, st);
  if (mx <= 2) return launch_a<2>(g, tl, H2, coil, A, xpart, nchunk, st);
  if (mx <= 4) return launch_a<4>(g, tl, H2, coil, A, xpart, nchunk, st);
  if (mx <= 8) return launch_a<8>(g, tl, H2, coil, A, xpart, nchunk, st);
  return cudaErrorInvalidValue;
}

}  // namespace gpjc
