// Device bodies of the FP32 register-tiled readout stage, shared by the
// single-slice kernels (k_readout_f.cu, k_readout_a.cu, k_readout_a2.cu)
// and the persistent batch kernel (k_batch.cu), and the forward kernel with
// batched readout transforms (k1f_batched, k_readout_f2.cu).
//
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
#pragma once
#include <algorithm>
#include <cstdlib>
#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kRThreads = 256;

// Preferred shared-memory carveout (percent of the maximum) of a readout
// kernel with `smem` bytes per block: just enough for the blocks its
// registers allow per SM, so the rest of the unified L1 / shared memory
// caches A_g and the factor tables (the forward kernel, limited to two
// blocks by its registers, gains ~5%; the adjoint keeps its three blocks).
// GPJC_READOUT_CARVEOUT (0..100) overrides it.
inline int readout_carveout(const void* func, size_t smem) {
  if (const char* e = getenv("GPJC_READOUT_CARVEOUT")) {
    const int c = atoi(e);
    if (c >= 0 && c <= 100) return c;
  }
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0;
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      fa.numRegs <= 0 || smem_sm <= 0) {
    cudaGetLastError();
    return 100;
  }
  const int by_regs = 65536 / (fa.numRegs * kRThreads);
  const size_t need = (size_t)std::max(by_regs, 1) * (smem + 1024);
  const int pct = (int)((need * 100 + (size_t)smem_sm - 1) / (size_t)smem_sm);
  return std::min(100, std::max(pct, 1));
}

// logical row stride of the spectra in shared memory (multiple of 8, so a
// row's padded sub-buffer starts at spad(r * stride))
__host__ __device__ inline int u_stride(int ntx) { return (ntx + 7) & ~7; }

// forward spectra U: two padding values every 8, so that a patch of 8 (or
// 16, ...) samples starts on a 16-byte boundary and pairs of samples can be
// read with one 16-byte load
__host__ __device__ inline int upad(int i) { return i + 2 * (i >> 3); }
__host__ __device__ inline int upad_size(int n) { return n + 2 * (n >> 3) + 2; }

// staged H2 rows, general layout: one padding slot every 16 columns
// (conflict-free when the tiles of a warp read columns 16 kept components
// apart, one component at a time)
__host__ __device__ inline int hpad(int i) { return i + (i >> 4); }
__host__ __device__ inline int hpad_size(int n) { return n + (n >> 4) + 1; }

// staged H2 rows, paired layout (RTiles::hpair: every patch offset on a
// 16-component boundary, even keep <= 16): element i at hswz(i).  Pairs
// (2q, 2q + 1) stay together
// (one 16-byte load) and the pair index q is XOR-swizzled in its low three
// bits by bits 3-5 and 10 of q: a permutation within each aligned block of 8
// pairs, under which the tiles of a warp (4 groups x 2 column blocks whose
// patches start 16 kept components apart, on a 32-group, keep-16 layout)
// read pairs in 8 different bank quads.
__host__ __device__ inline int hswz_sw(int q) { return ((q >> 3) ^ ((q >> 10) << 2)) & 7; }
__host__ __device__ inline int hswz(int i) {
  const int q = i >> 1;
  return ((q ^ hswz_sw(q)) << 1) | (i & 1);
}
__host__ __device__ inline int hswz_size(int n) { return (n + 15) & ~15; }


__device__ __forceinline__ float2 post_at(const Geo& g, int t, int row) {
  const int y = row % g.ny, z = row / g.ny;
  const float2 py = g.post_y[(size_t)y * g.ntx + t];
  if (g.nz == 1) return py;
  return cmul(py, g.post_z[(size_t)z * g.ntx + t]);
}

// Loads of data another stage of the same launch may have written use plain
// (coherent) loads when P is set (persistent batch kernel); read-only inputs
// always go through the read-only path.
template <bool P>
__device__ __forceinline__ float2 ldm(const float2* p) {
  if (P) return __ldcg(p);  // L2-coherent: written by another block of the same launch
  return __ldg(p);
}

// ------------------------------------------------------------------ forward --
// A_g contraction of one coil's spectra U (rows of the block, stride st,
// upad layout) into the register tiles: acc[m][c][k] += sum_tau
// A_g[k][nw + tau] U[uoff + tau] (Eq. 13).
template <int MAXT>
__device__ __forceinline__ void k1f_contract(float2 (&acc)[MAXT][4][4], const int4 (&hdr)[MAXT],
                                             const int (&uoff)[MAXT][4], const float2* U,
                                             const float2* __restrict__ AT, int nw, int w) {
#pragma unroll
  for (int m = 0; m < MAXT; ++m) {
    const int4 h = hdr[m];  // (aoff_g + k0, keep_g, kcnt, unused)
    if (h.z == 0) continue;
    const float2* Ap = AT + h.x + (size_t)nw * h.y;
    // full tiles with 16-byte aligned rows take two 16-byte loads per tau
    const bool vec = h.z == 4 && (h.y & 1) == 0 && (((uintptr_t)Ap) & 15) == 0;
    // patches on 8-sample boundaries: two samples per 16-byte load of U
    bool upair = vec && (w & 7) == 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) upair = upair && (uoff[m][c] < 0 || (uoff[m][c] & 7) == 0);
    if (upair) {
#pragma unroll 2
      for (int tau = 0; tau < w; tau += 2) {
        float2 a0[4], a1[4], u0[4], u1[4];
        {
          const float4 p01 = __ldg(reinterpret_cast<const float4*>(Ap));
          const float4 p23 = __ldg(reinterpret_cast<const float4*>(Ap + 2));
          const float4 q01 = __ldg(reinterpret_cast<const float4*>(Ap + h.y));
          const float4 q23 = __ldg(reinterpret_cast<const float4*>(Ap + h.y + 2));
          a0[0] = make_float2(p01.x, p01.y); a0[1] = make_float2(p01.z, p01.w);
          a0[2] = make_float2(p23.x, p23.y); a0[3] = make_float2(p23.z, p23.w);
          a1[0] = make_float2(q01.x, q01.y); a1[1] = make_float2(q01.z, q01.w);
          a1[2] = make_float2(q23.x, q23.y); a1[3] = make_float2(q23.z, q23.w);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (uoff[m][c] >= 0) v = *reinterpret_cast<const float4*>(U + upad(uoff[m][c] + tau));
          u0[c] = make_float2(v.x, v.y);
          u1[c] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            cfma(acc[m][c][k], a0[k], u0[c]);
            cfma(acc[m][c][k], a1[k], u1[c]);
          }
        Ap += 2 * h.y;
      }
      continue;
    }
    for (int tau = 0; tau < w; ++tau) {
      float2 a[4], u[4];
      if (vec) {
        const float4 a01 = __ldg(reinterpret_cast<const float4*>(Ap));
        const float4 a23 = __ldg(reinterpret_cast<const float4*>(Ap + 2));
        a[0] = make_float2(a01.x, a01.y);
        a[1] = make_float2(a01.z, a01.w);
        a[2] = make_float2(a23.x, a23.y);
        a[3] = make_float2(a23.z, a23.w);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = k < h.z ? __ldg(Ap + k) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) u[c] = uoff[m][c] >= 0 ? U[upad(uoff[m][c] + tau)] : make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) cfma(acc[m][c][k], a[k], u[c]);
      Ap += h.y;
    }
  }
}

template <int MAXT, bool P>
__device__ __forceinline__ void k1f_body(const Geo& g, const RTiles& tl, const float2* __restrict__ x,
                                         const float2* __restrict__ coil, const float2* __restrict__ AT,
                                         float2* __restrict__ Hpart, int cpc, int rblock, int chunk,
                                         float2* rsm) {
  const int rb = tl.rb, st = u_stride(g.ntx);
  float2* U = rsm;
  float2* A = U + upad_size(rb * st);
  float2* B = A + spad_size(g.ntx);
  float2* tw = B + spad_size(g.ntx);
  const int row0 = rblock * rb;
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
      float2* Ur = U + upad(r * st);
      const float2* py = g.post_y + (size_t)(row % g.ny) * g.ntx;
      const float2* pz = g.post_z + (size_t)(row / g.ny) * g.ntx;
      if (g.fx.n1 > 0) {
        // u = c_n x once per pixel; the two-pass FFT applies the pre-twiddle
        // while loading and the wave / centring factor while storing U
        for (int xx = threadIdx.x; xx < nx; xx += blockDim.x) A[xx] = cmul(__ldg(crow + xx), ldm<P>(xrow + xx));
        __syncthreads();
        auto ld = [&](int s, int xx) { return cmul(A[xx], __ldg(g.pre + s * nx + xx)); };
        auto stf = [&](int s, int m, float2 v) {
          const int t = m * os + s;
          float2 pt = __ldg(py + t);
          if (g.nz > 1) pt = cmul(pt, __ldg(pz + t));
          Ur[upad(t)] = cmul(v, pt);
        };
        fft2p_cb_dispatch<-1>(g.fx.n1, g.fx.n2, ld, stf, B, os, tw, threadIdx.x, blockDim.x);
      } else {
        // u = c_n x once per pixel, then its os pre-twiddled copies
        for (int xx = threadIdx.x; xx < nx; xx += blockDim.x) {
          const float2 u = cmul(__ldg(crow + xx), ldm<P>(xrow + xx));
          for (int s = 0; s < os; ++s) A[spad(s * nx + xx)] = cmul(u, __ldg(g.pre + s * nx + xx));
        }
        __syncthreads();
        float2* R = fft_stockham<-1, true>(A, B, os, nx, g.fx, tw, threadIdx.x, blockDim.x);
        for (int m = threadIdx.x; m < nx; m += blockDim.x)
          for (int s = 0; s < os; ++s) {
            const int t = m * os + s;
            float2 pt = __ldg(py + t);
            if (g.nz > 1) pt = cmul(pt, __ldg(pz + t));
            Ur[upad(t)] = cmul(R[spad(s * nx + m)], pt);
          }
        __syncthreads();
      }
    }
    k1f_contract<MAXT>(acc, hdr, uoff, U, AT, n * w, w);
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

template <int MAXT>
__global__ void __launch_bounds__(kRThreads) k1f_tiled(Geo g, RTiles tl, const float2* __restrict__ x,
                                                       const float2* __restrict__ coil,
                                                       const float2* __restrict__ AT, float2* __restrict__ Hpart,
                                                       int cpc) {
  extern __shared__ float2 rsm[];
  k1f_body<MAXT, false>(g, tl, x, coil, AT, Hpart, cpc, blockIdx.x, blockIdx.y, rsm);
}

// ------------------------------------------- forward, batched transforms --
// Two-pass readout lengths (g.fx.n1 > 0).  Coils are taken nb at a time: the
// os readout DFTs of every row of the block and of the nb coils run in one
// two-pass call (nb * nrows * os transforms, so that both passes give every
// thread a task where one row of one coil would leave most of them idle),
// then the A_g contraction reads the nb spectra into the same register
// tiles.  Three block barriers per nb coils: after c_n x, between the two
// passes, after the second pass; the contraction of one step needs none
// before the next step's c_n x, which writes a buffer the contraction does
// not read.
//
// Shared memory (readout_fwd2_smem): U, nb spectra buffers of the block's
// rows (upad layout, usz each); A, c_n x per (coil, row); B, the FFT
// scratch (nb * rb * ntx); the twiddle table.
__host__ __device__ inline int fwd2_usz(int rb, int ntx) { return (upad_size(rb * u_stride(ntx)) + 1) & ~1; }

// Balanced launch (units > 0): one wave of gridDim.x blocks; the
// (row block, coil group of nbmax coils) units, row-block-major, are split
// into gridDim.x contiguous ranges, so every block gets the same number of
// units to within one.  A range covers parts of several row blocks; each
// part (segment) sums its coils into its own plane of Hpart, numbered by the
// segment's position among the row block's segments (block boundaries
// B_j = floor(units j / gridDim.x) inside the row block), and the row
// block's last segment writes zeros to the planes the row block does not
// use, so the phase-encode stage sums `planes` planes in a fixed order.
template <int MAXT>
__global__ void __launch_bounds__(kRThreads) k1f_batched(Geo g, RTiles tl, const float2* __restrict__ x,
                                                         const float2* __restrict__ coil,
                                                         const float2* __restrict__ AT,
                                                         float2* __restrict__ Hpart, int cpc, int nbmax, int units,
                                                         int npair, int planes) {
  extern __shared__ float2 rsm[];
  const int rb = tl.rb, st = u_stride(g.ntx), usz = fwd2_usz(rb, g.ntx);
  const int nx = g.nx, os = g.os, w = g.w;
  float2* U = rsm;
  float2* A = U + nbmax * usz;
  float2* B = A + nbmax * rb * nx;
  float2* tw = B + nbmax * rb * g.ntx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * nx;

  // rows [row0, row0 + nrows), coils [n0, n1) into plane `plane`; zeros into
  // planes [zero0, planes)
  auto segment = [&](int row0, int n0, int n1, int plane, int zero0) {
    const int nrows = min(rb, g.rows - row0);
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
        uoff[m][c] = (cc.x >= 0 && cc.x / st < nrows) ? cc.x : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[m][c][k] = make_float2(0.f, 0.f);
      }
    }
    const int per = nrows * os;  // transforms per coil
    for (int n = n0; n < n1; n += nbmax) {
      const int nb = min(nbmax, n1 - n);
      // c_n x for the nb coils and the block's rows, [coil j][row r][x]
      const float2* xb = x + (size_t)row0 * nx;
      for (int i = threadIdx.x; i < nb * nrows * nx; i += blockDim.x) {
        const int j = i / (nrows * nx), rx = i - j * nrows * nx;
        A[i] = cmul(__ldg(coil + (size_t)(n + j) * L + (size_t)row0 * nx + rx), __ldg(xb + rx));
      }
      __syncthreads();
      // transform f = (j nrows + r) os + s: pre-twiddle s while loading, the
      // wave / centring factor of (row, t = m os + s) while storing U_j
      auto ld = [&](int f, int xx) {
        const int q = f / os, s = f - q * os;
        return cmul(A[q * nx + xx], __ldg(g.pre + s * nx + xx));
      };
      auto stf = [&](int f, int m, float2 v) {
        const int q = f / os, s = f - q * os, j = q / nrows, r = q - j * nrows;
        const int t = m * os + s;
        U[j * usz + upad(r * st + t)] = cmul(v, post_at(g, t, row0 + r));
      };
      fft2p_cb_dispatch<-1>(g.fx.n1, g.fx.n2, ld, stf, B, nb * per, tw, threadIdx.x, blockDim.x);
      for (int j = 0; j < nb; ++j) k1f_contract<MAXT>(acc, hdr, uoff, U + j * usz, AT, (n + j) * w, w);
    }
#pragma unroll
    for (int m = 0; m < MAXT; ++m) {
      const int tile = threadIdx.x + m * kRThreads;
      if (tile >= tl.nt) continue;
      const int kc = hdr[m].z;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (uoff[m][c] < 0) continue;
        const int o = tl.cols[tile * 4 + c].y;  // r * ntxc + off_p + k0
        float2* out = Hpart + ((size_t)plane * g.rows + row0) * g.ntxc + o;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < kc) out[k] = acc[m][c][k];
        for (int q = zero0; q < planes; ++q) {
          float2* z = Hpart + ((size_t)q * g.rows + row0) * g.ntxc + o;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (k < kc) z[k] = make_float2(0.f, 0.f);
        }
      }
    }
  };

  // one segment per block for the row-block x coil-chunk grid (units == 0)
  const long long G = gridDim.x, Uu = units > 0 ? units : 1;
  int u = units > 0 ? (int)(Uu * blockIdx.x / G) : 0;
  const int u1 = units > 0 ? (int)(Uu * (blockIdx.x + 1) / G) : 1;
  // boundaries B_j = floor(units j / G) at or below v: ceil((v + 1) G / units)
  auto cnt = [&](int v) { return (int)(((long long)(v + 1) * G + Uu - 1) / Uu); };
  while (u < u1) {
    int row0, n0, n1, plane, zero0, unext;
    if (units == 0) {
      row0 = blockIdx.x * rb;
      n0 = blockIdx.y * cpc;
      n1 = min(g.nc, n0 + cpc);
      plane = blockIdx.y;
      zero0 = planes;
      unext = u1;
    } else {
      const int rbk = u / npair;
      const int rs = rbk * npair, re = rs + npair;
      unext = min(u1, re);
      const int ord = cnt(u) - cnt(rs), nseg = 1 + cnt(re - 1) - cnt(rs);
      row0 = rbk * rb;
      n0 = (u - rs) * nbmax;
      n1 = min(g.nc, (unext - rs) * nbmax);
      plane = ord;
      zero0 = ord == nseg - 1 ? nseg : planes;
    }
    segment(row0, n0, n1, plane, zero0);
    u = unext;
  }
}

// ------------------------------------------------------------------ adjoint --
// A_g^H on every tile of the block for coil n (Eq. 15): U_r[t] = sum_k
// conj(A_g[k][n w + tau]) H2[row][off_p + k], TS samples x 4 columns per
// tile, written to U (rows of the block, stride st, spad layout): in natural
// order t for two-pass lengths (the FFT applies the wave / centring factor
// while loading), else times conj(post) at s nx + m for the Stockham FFT.
template <bool P, int TS>
__device__ __forceinline__ void k1a_contract(const Geo& g, const RTiles& tl, const float2* __restrict__ H2,
                                             const float2* Hs, bool hs, const float2* __restrict__ Arow, int n,
                                             int row0, int nrows, int st, float2* U) {
  const int nx = g.nx, os = g.os, w = g.w, ns = g.ns;
  // A^H on every tile: U_r[t] = sum_k conj(A_g[k][n w + tau]) H2[row][off_p + k]
  // (TS samples x 4 columns per tile); the tile descriptors are re-read
  // (L1) to keep registers for the sums
  for (int tile = threadIdx.x; tile < tl.nt; tile += kRThreads) {
    const int4 h = tl.hdr[tile];  // (aoff_g + tau0, keep_g, tcnt, unused)
    int cr[4], hoff[4];
    const float2* hp[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int4 cc = tl.cols[tile * 4 + c];  // (r, off_p, p w + tau0, 0)
      cr[c] = (cc.x >= 0 && cc.x < nrows) ? cc.x : -1;
      hp[c] = cr[c] >= 0 ? H2 + (size_t)(row0 + cc.x) * g.ntxc + cc.y : H2;
      hoff[c] = cr[c] >= 0 ? cc.x * g.ntxc + cc.y : 0;
    }
    float2 acc[4][TS];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < TS; ++k) acc[c][k] = make_float2(0.f, 0.f);
    const float2* Ap = Arow + h.x + n * w;
    // full tiles with 16-byte aligned rows load two samples at a time
    const bool vec = h.z == TS && (ns & 1) == 0 && (((uintptr_t)Ap) & 15) == 0;
    // paired staging, full tiles, columns on 16-component boundaries and an
    // even keep <= 16: the components of a column lie in one swizzle block of
    // 8 pairs, where pair k/2 sits at hoff + (k ^ hx) (hswz), so they are read
    // in pairs, one 16-byte load per column and pair
    const bool sw = hs && tl.hpair;
    bool pairs = vec && sw && h.y <= 16 && (h.y & 1) == 0;
    int hx[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pairs = pairs && cr[c] >= 0 && (hoff[c] & 15) == 0;
      hx[c] = 2 * hswz_sw(hoff[c] >> 1);
    }
    if (pairs) {
#pragma unroll 1
      for (int k = 0; k < h.y; k += 2) {
        float2 a0[TS], a1[TS], h0[4], h1[4];
#pragma unroll
        for (int tt = 0; tt < TS; tt += 2) {
          const float4 v0 = __ldg(reinterpret_cast<const float4*>(Ap + tt));
          const float4 v1 = __ldg(reinterpret_cast<const float4*>(Ap + ns + tt));
          a0[tt] = make_float2(v0.x, v0.y);
          a0[tt + 1] = make_float2(v0.z, v0.w);
          a1[tt] = make_float2(v1.x, v1.y);
          a1[tt + 1] = make_float2(v1.z, v1.w);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(Hs + hoff[c] + (k ^ hx[c]));
          h0[c] = make_float2(v.x, v.y);
          h1[c] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int tt = 0; tt < TS; ++tt) {
            cfmac(acc[c][tt], a0[tt], h0[c]);
            cfmac(acc[c][tt], a1[tt], h1[c]);
          }
        Ap += 2 * ns;
      }
    }
#pragma unroll 2
    for (int k = 0; !pairs && k < h.y; ++k) {
      float2 a[TS], hv[4];
      if (vec) {
#pragma unroll
        for (int tt = 0; tt < TS; tt += 2) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(Ap + tt));
          a[tt] = make_float2(v.x, v.y);
          a[tt + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int tt = 0; tt < TS; ++tt) a[tt] = tt < h.z ? __ldg(Ap + tt) : make_float2(0.f, 0.f);
      }
      if (sw) {
#pragma unroll
        for (int c = 0; c < 4; ++c) hv[c] = cr[c] >= 0 ? Hs[hswz(hoff[c] + k)] : make_float2(0.f, 0.f);
      } else if (hs) {
#pragma unroll
        for (int c = 0; c < 4; ++c) hv[c] = cr[c] >= 0 ? Hs[hpad(hoff[c] + k)] : make_float2(0.f, 0.f);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) hv[c] = cr[c] >= 0 ? ldm<P>(hp[c] + k) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int tt = 0; tt < TS; ++tt) cfmac(acc[c][tt], a[tt], hv[c]);
      Ap += ns;
    }
    const bool two = g.fx.n1 > 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (cr[c] < 0) continue;
      float2* Ur = U + spad(cr[c] * st);
      const int t0 = tl.cols[tile * 4 + c].z;
      if (two) {
        // natural order t; the FFT applies the wave / centring factor while loading
#pragma unroll
        for (int tt = 0; tt < TS; ++tt)
          if (tt < h.z) Ur[spad(t0 + tt)] = acc[c][tt];
        continue;
      }
      const int row = row0 + cr[c];
      const float2* py = g.post_y + (size_t)(row % g.ny) * g.ntx;
      const float2* pz = g.post_z + (size_t)(row / g.ny) * g.ntx;
#pragma unroll
      for (int tt = 0; tt < TS; ++tt) {
        if (tt >= h.z) continue;
        const int t = t0 + tt;
        const int mm = t / os, s = t - mm * os;
        float2 pt = __ldg(py + t);
        if (g.nz > 1) pt = cmul(pt, __ldg(pz + t));
        Ur[spad(s * nx + mm)] = cmulc(pt, acc[c][tt]);
      }
    }
  }
}

template <int MAXX, bool P, int TS>
__device__ __forceinline__ void k1a_body(const Geo& g, const RTiles& tl, const float2* __restrict__ H2,
                                         const float2* __restrict__ coil, const float2* __restrict__ Arow,
                                         float2* __restrict__ xpart, int cpc, int rblock, int chunk,
                                         float2* rsm) {
  const int rb = tl.rb, st = u_stride(g.ntx);
  float2* U = rsm;
  float2* B = U + spad_size(rb * st);
  float2* tw = B + spad_size(g.ntx);
  float2* Hs = tw + g.nx;  // staged H2 rows (tl.hstage), 16-byte aligned (one spare slot)
  if (reinterpret_cast<uintptr_t>(Hs) & 15) ++Hs;
  const int row0 = rblock * rb;
  const int nrows = min(rb, g.rows - row0);
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) tw[i] = g.tw_x[i];
  const size_t L = (size_t)g.rows * g.nx;
  const int nx = g.nx, os = g.os;
  const bool hs = tl.hstage != 0;
  if (hs) {
    // the block's rows of H2, read once for all coils of the chunk
    const float2* src = H2 + (size_t)row0 * g.ntxc;
    if (tl.hpair)
      for (int i = threadIdx.x; i < nrows * g.ntxc; i += blockDim.x) Hs[hswz(i)] = ldm<P>(src + i);
    else
      for (int i = threadIdx.x; i < nrows * g.ntxc; i += blockDim.x) Hs[hpad(i)] = ldm<P>(src + i);
  }

  float2 xacc[MAXX];
#pragma unroll
  for (int j = 0; j < MAXX; ++j) xacc[j] = make_float2(0.f, 0.f);
  __syncthreads();
  const int n0 = chunk * cpc, n1 = min(g.nc, n0 + cpc);
  for (int n = n0; n < n1; ++n) {
    k1a_contract<P, TS>(g, tl, H2, Hs, hs, Arow, n, row0, nrows, st, U);
    __syncthreads();
    for (int r = 0; r < nrows; ++r) {
      float2* Ur = U + spad(r * st);
      const float2* R;
      if (g.fx.n1 > 0) {
        const int row = row0 + r;
        const float2* py = g.post_y + (size_t)(row % g.ny) * g.ntx;
        const float2* pz = g.post_z + (size_t)(row / g.ny) * g.ntx;
        auto ld = [&](int s, int m) {
          const int t = m * os + s;
          float2 pt = __ldg(py + t);
          if (g.nz > 1) pt = cmul(pt, __ldg(pz + t));
          return cmulc(pt, Ur[spad(t)]);
        };
        // the row's spectra are consumed by the first pass: the result
        // overwrites them in natural order (transform s at s nx)
        auto stf = [&](int s, int xx, float2 v) { Ur[s * nx + xx] = v; };
        fft2p_cb_dispatch<+1>(g.fx.n1, g.fx.n2, ld, stf, B, os, tw, threadIdx.x, blockDim.x);
        R = Ur;
      } else {
        R = fft_stockham<+1, true>(Ur, B, os, nx, g.fx, tw, threadIdx.x, blockDim.x);
      }
      const bool padr = g.fx.n1 == 0;
      const float2* crow = coil + n * L + (size_t)(row0 + r) * nx;
      // thread-owned output slots (r', x) = slot / nx, slot % nx
#pragma unroll
      for (int j = 0; j < MAXX; ++j) {
        const int slot = threadIdx.x + j * kRThreads;
        if (slot < nrows * nx && slot / nx == r) {
          const int xx = slot - r * nx;
          float2 u = make_float2(0.f, 0.f);
          for (int s = 0; s < os; ++s) {
            const int i = s * nx + xx;
            cfmac(u, __ldg(g.pre + i), R[padr ? spad(i) : i]);
          }
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

// (register budgets for 3 blocks per SM with two-sample tiles, whose shared
// memory fits three blocks beside the staged H2 row, and 2 with four-sample
// tiles)
template <int MAXX, int TS>
__global__ void __launch_bounds__(kRThreads, TS == 2 ? 3 : 2) k1a_tiled(Geo g, RTiles tl, const float2* __restrict__ H2,
                                                       const float2* __restrict__ coil,
                                                       const float2* __restrict__ Arow, float2* __restrict__ xpart,
                                                       int cpc) {
  extern __shared__ float2 rsm[];
  k1a_body<MAXX, false, TS>(g, tl, H2, coil, Arow, xpart, cpc, blockIdx.x, blockIdx.y, rsm);
}

}  // namespace gpjc
