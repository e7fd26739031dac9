// Device-side helpers shared by the gpjc kernels: complex arithmetic, a
// mixed-radix (2,3,4,5,7,8) Stockham FFT in shared memory, block reductions
// and the deterministic "last block finishes" grid reduction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpjc_internal.h"

namespace gpjc {

// ------------------------------------------------------------ complex --
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
// e^{i pi a}
__device__ __forceinline__ float2 expipi(float a) {
  float s, c;
  sincospif(a, &s, &c);
  return make_float2(c, s);
}

// ------------------------------------------------------------ small DFTs --
// In-register R-point DFT, X[q] = sum_r v[r] exp(SIGN * 2 pi i r q / R).
template <int SIGN>
__device__ __forceinline__ float2 mul_sign_i(float2 a) {
  // multiply by SIGN * i
  return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2* v) {
  float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  float2 b0 = cadd(v[1], v[3]), b1 = mul_sign_i<SIGN>(csub(v[1], v[3]));
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[3] = csub(a1, b1);
}

template <int SIGN>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<SIGN>(e);
  dft4<SIGN>(o);
  const float h = 0.70710678118654752440f;
  // twiddles W8^k, W8 = exp(SIGN 2 pi i / 8)
  float2 w1 = make_float2(h, SIGN * h);
  float2 w3 = make_float2(-h, SIGN * h);
  float2 t0 = o[0];
  float2 t1 = cmul(o[1], w1);
  float2 t2 = mul_sign_i<SIGN>(o[2]);
  float2 t3 = cmul(o[3], w3);
  v[0] = cadd(e[0], t0);
  v[4] = csub(e[0], t0);
  v[1] = cadd(e[1], t1);
  v[5] = csub(e[1], t1);
  v[2] = cadd(e[2], t2);
  v[6] = csub(e[2], t2);
  v[3] = cadd(e[3], t3);
  v[7] = csub(e[3], t3);
}

// Direct odd-radix DFT from cos / sin of 2 pi k / R.
template <int R, int SIGN>
__device__ __forceinline__ void dft_odd(float2* v, const float* c, const float* s) {
  float2 out[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    float2 acc = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int m = (r * q) % R;
      float2 w = make_float2(c[m], SIGN * s[m]);
      cfma(acc, v[r], w);
    }
    out[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = out[q];
}

template <int SIGN>
__device__ __forceinline__ void dft3(float2* v) {
  const float c[3] = {1.0f, -0.5f, -0.5f};
  const float s[3] = {0.0f, 0.86602540378443865f, -0.86602540378443865f};
  dft_odd<3, SIGN>(v, c, s);
}
template <int SIGN>
__device__ __forceinline__ void dft5(float2* v) {
  const float c[5] = {1.0f, 0.30901699437494742f, -0.80901699437494742f, -0.80901699437494742f,
                      0.30901699437494742f};
  const float s[5] = {0.0f, 0.95105651629515357f, 0.58778525229247313f, -0.58778525229247313f,
                      -0.95105651629515357f};
  dft_odd<5, SIGN>(v, c, s);
}
template <int SIGN>
__device__ __forceinline__ void dft7(float2* v) {
  const float c[7] = {1.0f, 0.62348980185873353f, -0.22252093395631440f, -0.90096886790241913f,
                      -0.90096886790241913f, -0.22252093395631440f, 0.62348980185873353f};
  const float s[7] = {0.0f, 0.78183148246802981f, 0.97492791218182361f, 0.43388373911755812f,
                      -0.43388373911755812f, -0.97492791218182361f, -0.78183148246802981f};
  dft_odd<7, SIGN>(v, c, s);
}

// Shared-memory index with one padding slot every 8 complex values: keeps
// the stride-R stores of the first Stockham stages (R = 2..8) and the
// stride-8 pattern after a radix-8 stage free of bank conflicts.
__device__ __forceinline__ int spad(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int spad_size(int n) { return n + (n >> 3) + 1; }

// One Stockham stage of radix R on `batch` contiguous transforms of length n.
// tw[k] = exp(-2 pi i k / n) for k < n.  With PAD, element i of the logical
// buffer lives at spad(i).
template <int R, int SIGN, bool PAD = false>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               int n, int batch, int bs, int ns,
                                               const float2* __restrict__ tw, int tid, int nthr) {
  const int m = n / R;
  const int total = batch * m;
  const int twstep = n / (ns * R);
  for (int idx = tid; idx < total; idx += nthr) {
    const int f = idx / m;
    const int j = idx - f * m;
    const int sb = f * bs;
    float2 v[R];
    const int jq = j / ns;
    const int k = j - jq * ns;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int li = sb + j + r * m;
      float2 a = src[PAD ? spad(li) : li];
      if (r > 0 && k > 0) {
        const int e = k * r * twstep;  // < n since k < ns and r < R
        float2 w = tw[e];
        if (SIGN > 0) w.y = -w.y;
        a = cmul(a, w);
      }
      v[r] = a;
    }
    if (R == 2) dft2<SIGN>(v);
    if (R == 3) dft3<SIGN>(v);
    if (R == 4) dft4<SIGN>(v);
    if (R == 5) dft5<SIGN>(v);
    if (R == 7) dft7<SIGN>(v);
    if (R == 8) dft8<SIGN>(v);
    const int base = sb + jq * ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int lo = base + q * ns;
      dst[PAD ? spad(lo) : lo] = v[q];
    }
  }
}

// Batched ping-pong Stockham FFT (unnormalised) of `batch` transforms whose
// starts are `bs` elements apart.  Data starts in `a`; returns the buffer
// holding the result (a or b).  SIGN = -1 forward, +1 inverse.  Must be
// called by all threads of the block; ends with __syncthreads().
template <int SIGN, bool PAD = false>
__device__ float2* fft_stockham(float2* a, float2* b, int batch, int bs, const FftPlan& pl,
                                const float2* __restrict__ tw, int tid, int nthr) {
  int ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.rad[st];
    switch (R) {
      case 2: stockham_stage<2, SIGN, PAD>(a, b, pl.n, batch, bs, ns, tw, tid, nthr); break;
      case 3: stockham_stage<3, SIGN, PAD>(a, b, pl.n, batch, bs, ns, tw, tid, nthr); break;
      case 4: stockham_stage<4, SIGN, PAD>(a, b, pl.n, batch, bs, ns, tw, tid, nthr); break;
      case 5: stockham_stage<5, SIGN, PAD>(a, b, pl.n, batch, bs, ns, tw, tid, nthr); break;
      case 7: stockham_stage<7, SIGN, PAD>(a, b, pl.n, batch, bs, ns, tw, tid, nthr); break;
      default: stockham_stage<8, SIGN, PAD>(a, b, pl.n, batch, bs, ns, tw, tid, nthr); break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    ns *= R;
  }
  return a;
}

}  // namespace gpjc
#include "gpjc_fft.cuh"
namespace gpjc {

// Batched FFT of `batch` transforms of length pl.n (starts `bs` apart, data in
// `a`, scratch `b`; returns the buffer with the result).  Lengths with a
// two-pass plan (pl.n1 > 0; the table `tw` then holds exp(-2 pi i i2 k1 / n)
// at k1 n2 + i2) run the register two-pass kernel, the others the radix
// stages (`tw` holds exp(-2 pi i k / n)).  Must be called by all threads of
// the block; ends with __syncthreads().
template <int SIGN, bool PAD = false>
__device__ __forceinline__ float2* fft_batch(float2* a, float2* b, int batch, int bs, const FftPlan& pl,
                                             const float2* __restrict__ tw, int tid, int nthr) {
  if (pl.n1 > 0 && fft2p_dispatch<SIGN, PAD>(pl.n1, pl.n2, a, b, batch, bs, tw, tid, nthr)) return a;
  return fft_stockham<SIGN, PAD>(a, b, batch, bs, pl, tw, tid, nthr);
}

// ------------------------------------------------------------ reductions --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; result valid in thread 0.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double r = 0.0;
  if (wid == 0) {
    r = lane < nw ? red[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Grid reduction with a deterministic final sum: every block stores its
// partial, the last block to arrive sums all partials in block order and
// stores the result in *out (then re-arms the counter).  Returns true in the
// one thread that wrote *out.
__device__ __forceinline__ bool grid_sum_finalize(double v, double* partials, unsigned* counter,
                                                  double* out, double* red) {
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  double s = block_sum(v, red);
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[bid] = s;
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc = 0.0;
  // fixed-order sum: thread t sums partials t, t+blockDim, ... ; then the
  // block tree combines them in a fixed pattern.
  for (unsigned i = threadIdx.x; i < nblk; i += blockDim.x) acc += ((volatile double*)partials)[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    *out = acc;
    *counter = 0u;
    return true;
  }
  return false;
}

// ------------------------------------------------------------------ phase-encode (2D) --
// A block owns kPeCB columns of the hybrid matrix [ny][ncols].  Centred
// unitary DFT along y: F[ky,y] = (-1)^y (-1)^{ky + ny/2} e^{-2 pi i ky y/ny} / sqrt(ny).
constexpr int kPeCB = 8;  // equal to kCB of k_pe.cu
__device__ __forceinline__ float pe_sgn(int k) { return (k & 1) ? -1.0f : 1.0f; }

// H = F_y^H M^T Sc for the columns of block `cb`.
__device__ __forceinline__ void pe_adj2d_body(const Geo& g, const float2* __restrict__ Sc, int ncols,
                                              float2* __restrict__ H, int cb, float2* smem) {
  const int ny = g.ny, bs = ny + 1;
  float2* a = smem;
  float2* b = smem + kPeCB * bs;
  float2* tw = smem + 2 * kPeCB * bs;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = g.tw_y[i];
  for (int i = threadIdx.x; i < kPeCB * bs; i += blockDim.x) a[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int col0 = cb * kPeCB;
  for (int i = threadIdx.x; i < g.n_lines * kPeCB; i += blockDim.x) {
    const int l = i / kPeCB, c = i - l * kPeCB;
    const int col = col0 + c;
    if (col < ncols) {
      const int ky = g.line_ky[l];
      a[c * bs + ky] = cscale(__ldg(Sc + (size_t)l * ncols + col), pe_sgn(ky + ny / 2) * g.inv_sqrt_ny);
    }
  }
  __syncthreads();
  float2* res = fft_batch<+1>(a, b, kPeCB, bs, g.fy, tw, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < ny * kPeCB; i += blockDim.x) {
    const int y = i / kPeCB, c = i - y * kPeCB;
    const int col = col0 + c;
    if (col < ncols) H[(size_t)y * ncols + col] = cscale(res[c * bs + y], pe_sgn(y));
  }
  __syncthreads();
}

// H2 = F_y^H M^T M F_y (sum over chunks of Hpart) for the columns of block
// `cb`; returns the block's ||M F_y H||^2 (valid in thread 0).  With P the
// hybrid partials are read with coherent loads.
template <bool P>
__device__ __forceinline__ double pe_normal2d_body(const Geo& g, const float2* __restrict__ Hpart, int nchunk,
                                                   int ncols, float2* __restrict__ H2, int cb, float2* smem) {
  __shared__ double red[32];
  const int ny = g.ny, bs = ny + 1;
  float2* a = smem;
  float2* b = smem + kPeCB * bs;
  float2* tw = smem + 2 * kPeCB * bs;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = g.tw_y[i];
  const int col0 = cb * kPeCB;
  const size_t plane = (size_t)g.rows * ncols;
  for (int i = threadIdx.x; i < ny * kPeCB; i += blockDim.x) {
    const int y = i / kPeCB, c = i - y * kPeCB;
    const int col = col0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (col < ncols)
      for (int ch = 0; ch < nchunk; ++ch) {
        const float2* src = Hpart + ch * plane + (size_t)y * ncols + col;
        v = cadd(v, P ? __ldcg(src) : __ldg(src));
      }
    a[c * bs + y] = cscale(v, pe_sgn(y));
  }
  __syncthreads();
  float2* res = fft_batch<-1>(a, b, kPeCB, bs, g.fy, tw, threadIdx.x, blockDim.x);
  float2* oth = (res == a) ? b : a;
  const float inv_ny = 1.0f / (float)ny;
  double part = 0.0;
  for (int i = threadIdx.x; i < ny * kPeCB; i += blockDim.x) {
    const int c = i / ny, ky = i - c * ny;
    float2 v = res[c * bs + ky];
    if (g.line_of[ky] >= 0 && col0 + c < ncols) {
      part += ((double)v.x * v.x + (double)v.y * v.y) * inv_ny;
      v = cscale(v, inv_ny);
    } else {
      v = make_float2(0.f, 0.f);
    }
    res[c * bs + ky] = v;
  }
  __syncthreads();
  float2* res2 = fft_batch<+1>(res, oth, kPeCB, bs, g.fy, tw, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < ny * kPeCB; i += blockDim.x) {
    const int y = i / kPeCB, c = i - y * kPeCB;
    const int col = col0 + c;
    if (col < ncols) H2[(size_t)y * ncols + col] = cscale(res2[c * bs + y], pe_sgn(y));
  }
  const double tot = block_sum(part, red);
  __syncthreads();
  return tot;
}

}  // namespace gpjc
