// Reconstruction kernels (Sec. 3.4): CG on E_c^H E_c x = E_c^H S' (Eq. 16)
// and FISTA with an orthonormal Haar l1 term (Eq. 17, lambda_TV = 0).
//
// Vectors are FP32 complex; every inner product is accumulated in FP64 and
// reduced across the grid deterministically (the last block to finish sums
// the per-block partials in block order).  The CG scalars live in device
// memory so the whole loop runs without host synchronisation and can be
// captured in a CUDA graph.
//
// The Haar transform with J levels acts independently on each 2^J x 2^J
// tile of a slice (level j combines 2^j x 2^j pixel blocks), so the FISTA
// proximal step W^H soft(W z) is one tile-local kernel fused with the
// gradient step and the momentum update.
#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 1184;  // 152 SMs x 8 blocks

int sum_parts_blocks(size_t L) {
  size_t nb = (L + kVecThreads - 1) / kVecThreads;
  return (int)(nb < (size_t)kVecBlocks ? nb : (size_t)kVecBlocks);
}

// out = sum_c parts[c]; optional ||out||^2 into *nrm2.
__global__ void k_sum_parts(const float2* __restrict__ parts, int nchunk, size_t L, float2* __restrict__ out,
                            double* partials, unsigned* counter, double* nrm2) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x) {
    float2 v = parts[i];
    for (int c = 1; c < nchunk; ++c) v = cadd(v, parts[c * L + i]);
    out[i] = v;
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  if (nrm2) grid_sum_finalize(s, partials, counter, nrm2, red);
}

cudaError_t launch_sum_parts(const float2* parts, int nchunk, size_t L, float2* out, double* partials,
                             unsigned* counter, double* nrm2, cudaStream_t st) {
  note_launches(1); k_sum_parts<<<sum_parts_blocks(L), kVecThreads, 0, st>>>(parts, nchunk, L, out, partials, counter, nrm2);
  return cudaGetLastError();
}

// alpha = rr / qq; x += alpha p; r -= alpha (sum_c parts); rr_new = ||r||^2.
// rr == 0 leaves x and r unchanged (CG has converged exactly).
__global__ void k_cg_update1(const float2* __restrict__ parts, int nchunk, size_t L, float2* __restrict__ x,
                             float2* __restrict__ r, const float2* __restrict__ p, const double* rr,
                             const double* qq, double* partials, unsigned* counter, double* rr_new,
                             double* hist, int* status) {
  __shared__ double red[32];
  const double rrv = *rr, qqv = *qq;
  double alpha = (rrv == 0.0) ? 0.0 : rrv / qqv;
  if (!isfinite(alpha)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(status, (int)kDevNonFinite);
    alpha = 0.0;
  }
  const float a = (float)alpha;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x) {
    float2 ap = parts[i];
    for (int c = 1; c < nchunk; ++c) ap = cadd(ap, parts[c * L + i]);
    const float2 pv = p[i];
    float2 xv = x[i], rv = r[i];
    xv.x = fmaf(a, pv.x, xv.x);
    xv.y = fmaf(a, pv.y, xv.y);
    rv.x = fmaf(-a, ap.x, rv.x);
    rv.y = fmaf(-a, ap.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    s += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  if (grid_sum_finalize(s, partials, counter, rr_new, red)) {
    if (hist) *hist = *rr_new;
  }
}

cudaError_t launch_cg_update1(const float2* parts, int nchunk, size_t L, float2* x, float2* r, const float2* p,
                              const double* rr, const double* qq, double* partials, unsigned* counter,
                              double* rr_new, double* hist, int* status, cudaStream_t st) {
  note_launches(1); k_cg_update1<<<sum_parts_blocks(L), kVecThreads, 0, st>>>(parts, nchunk, L, x, r, p, rr, qq, partials,
                                                            counter, rr_new, hist, status);
  return cudaGetLastError();
}

// beta = rr_new / rr; p = r + beta p
__global__ void k_cg_update2(float2* __restrict__ p, const float2* __restrict__ r, size_t L, const double* rr,
                             const double* rr_new) {
  const double rrv = *rr;
  double beta = (rrv == 0.0) ? 0.0 : *rr_new / rrv;
  if (!isfinite(beta)) beta = 0.0;
  const float bt = (float)beta;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x) {
    if (rrv == 0.0) break;
    const float2 rv = r[i];
    float2 pv = p[i];
    pv.x = fmaf(bt, pv.x, rv.x);
    pv.y = fmaf(bt, pv.y, rv.y);
    p[i] = pv;
  }
}

cudaError_t launch_cg_update2(float2* p, const float2* r, size_t L, const double* rr, const double* rr_new,
                              cudaStream_t st) {
  note_launches(1); k_cg_update2<<<sum_parts_blocks(L), kVecThreads, 0, st>>>(p, r, L, rr, rr_new);
  return cudaGetLastError();
}

__global__ void k_axpby(float2* __restrict__ y, const float2* __restrict__ a, const float2* __restrict__ b,
                        float alpha, float beta, size_t L) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x) {
    const float2 av = a[i];
    const float2 bv = b ? b[i] : make_float2(0.f, 0.f);
    y[i] = make_float2(alpha * av.x + beta * bv.x, alpha * av.y + beta * bv.y);
  }
}

cudaError_t launch_axpby(float2* y, const float2* a, const float2* b, float alpha, float beta, size_t L,
                         cudaStream_t st) {
  note_launches(1); k_axpby<<<sum_parts_blocks(L), kVecThreads, 0, st>>>(y, a, b, alpha, beta, L);
  return cudaGetLastError();
}

// v = src / sqrt(*nrm2); optionally *Lout = sqrt(*nrm2) (power iteration).
__global__ void k_scale_by(float2* __restrict__ v, const float2* __restrict__ src, const double* nrm2, size_t L,
                           double* Lout) {
  const double n = sqrt(*nrm2);
  const float inv = n > 0.0 ? (float)(1.0 / n) : 0.0f;
  if (Lout && blockIdx.x == 0 && threadIdx.x == 0) *Lout = n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x)
    v[i] = cscale(src[i], inv);
}

cudaError_t launch_scale_by(float2* v, const float2* src, const double* nrm2, size_t L, double* Lout,
                            cudaStream_t st) {
  note_launches(1); k_scale_by<<<sum_parts_blocks(L), kVecThreads, 0, st>>>(v, src, nrm2, L, Lout);
  return cudaGetLastError();
}

__global__ void k_set_scalar(double* d, double v) { *d = v; }
cudaError_t launch_set_scalar(double* d, double v, cudaStream_t st) {
  note_launches(1); k_set_scalar<<<1, 1, 0, st>>>(d, v);
  return cudaGetLastError();
}

__global__ void k_copy(float2* __restrict__ d, const float2* __restrict__ s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}
__global__ void k_zero(float2* __restrict__ d, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = make_float2(0.f, 0.f);
}
cudaError_t launch_copy(float2* dst, const float2* src, size_t n, cudaStream_t st) {
  note_launches(1); k_copy<<<sum_parts_blocks(n), kVecThreads, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}
cudaError_t launch_zero(float2* dst, size_t n, cudaStream_t st) {
  note_launches(1); k_zero<<<sum_parts_blocks(n), kVecThreads, 0, st>>>(dst, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ per-set CG --
// Hybrid-space reconstruction (Sec. 3.4, algorithm #1): the normal
// equations decouple over the aliased sets of the mask (the phase-encode
// projection F^H M^T M F is block-diagonal over them), so each set runs its
// own CG on its rows with its own scalars alpha_Y, beta_Y.  The normal
// operator is applied to all rows at once (it does not couple the sets);
// the scalars are FP64 sums over each set's rows: one block per row forms
// the row's sum, and one block adds the rows of every set in the order of
// its member list (deterministic).

// v = sum_c parts[c] (row r, written to out when out != nullptr);
// rowval[r] = Re <a_r, v_r>  (a == nullptr: ||v_r||^2)
__global__ void __launch_bounds__(kVecThreads) k_ds_rowdot(const float2* __restrict__ parts, int nchunk, size_t L,
                                                          int nx, float2* __restrict__ out,
                                                          const float2* __restrict__ a, double* __restrict__ rowval) {
  __shared__ double red[32];
  const size_t base = (size_t)blockIdx.x * nx;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    float2 v = parts[base + i];
    for (int c = 1; c < nchunk; ++c) v = cadd(v, parts[c * L + base + i]);
    if (out) out[base + i] = v;
    const float2 u = a ? a[base + i] : v;
    acc += (double)u.x * v.x + (double)u.y * v.y;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) rowval[blockIdx.x] = acc;
}

// out[s] = sum of rowval over the rows of set s (member-list order);
// total (optional) = sum over all sets
__global__ void __launch_bounds__(kVecThreads) k_ds_setsum(const double* __restrict__ rowval, const int* __restrict__ ptr,
                                                          const int* __restrict__ rows, int n_sets,
                                                          double* __restrict__ out, double* total) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int s = threadIdx.x; s < n_sets; s += blockDim.x) {
    double v = 0.0;
    for (int i = ptr[s]; i < ptr[s + 1]; ++i) v += rowval[rows[i]];
    out[s] = v;
    acc += v;
  }
  acc = block_sum(acc, red);
  if (total && threadIdx.x == 0) *total = acc;
}

// per row r of set s = set_of_row[r]: alpha = rr[s] / pap[s] (0 when
// rr[s] == 0); x += alpha p; r -= alpha q; rowval[r] = ||r_r||^2
__global__ void __launch_bounds__(kVecThreads) k_ds_update1(int nx, const int* __restrict__ set_of_row,
                                                           float2* __restrict__ x, float2* __restrict__ r,
                                                           const float2* __restrict__ p, const float2* __restrict__ q,
                                                           const double* __restrict__ rr, const double* __restrict__ pap,
                                                           double* __restrict__ rowval, int* status) {
  __shared__ double red[32];
  const int s = set_of_row[blockIdx.x];
  const double rrv = rr[s];
  double alpha = rrv == 0.0 ? 0.0 : rrv / pap[s];
  if (!isfinite(alpha)) {
    if (threadIdx.x == 0) atomicExch(status, (int)kDevNonFinite);
    alpha = 0.0;
  }
  const float af = (float)alpha;
  const size_t base = (size_t)blockIdx.x * nx;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const float2 pv = p[base + i], qv = q[base + i];
    float2 xv = x[base + i], rv = r[base + i];
    xv.x = fmaf(af, pv.x, xv.x);
    xv.y = fmaf(af, pv.y, xv.y);
    rv.x = fmaf(-af, qv.x, rv.x);
    rv.y = fmaf(-af, qv.y, rv.y);
    x[base + i] = xv;
    r[base + i] = rv;
    acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) rowval[blockIdx.x] = acc;
}

// per row: beta = rr_new[s] / rr[s] (0 when rr[s] == 0); p = r + beta p
__global__ void __launch_bounds__(kVecThreads) k_ds_update2(int nx, const int* __restrict__ set_of_row,
                                                           float2* __restrict__ p, const float2* __restrict__ r,
                                                           const double* __restrict__ rr,
                                                           const double* __restrict__ rr_new) {
  const int s = set_of_row[blockIdx.x];
  const double rrv = rr[s];
  if (rrv == 0.0) return;  // converged set: p is not used again
  double beta = rr_new[s] / rrv;
  if (!isfinite(beta)) beta = 0.0;
  const float bf = (float)beta;
  const size_t base = (size_t)blockIdx.x * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const float2 rv = r[base + i];
    float2 pv = p[base + i];
    pv.x = fmaf(bf, pv.x, rv.x);
    pv.y = fmaf(bf, pv.y, rv.y);
    p[base + i] = pv;
  }
}

cudaError_t launch_ds_rowdot(const float2* parts, int nchunk, size_t L, int rows, int nx, float2* out,
                             const float2* a, double* rowval, cudaStream_t st) {
  note_launches(1); k_ds_rowdot<<<rows, kVecThreads, 0, st>>>(parts, nchunk, L, nx, out, a, rowval);
  return cudaGetLastError();
}
cudaError_t launch_ds_setsum(const double* rowval, const int* ptr, const int* rows, int n_sets, double* out,
                             double* total, cudaStream_t st) {
  note_launches(1); k_ds_setsum<<<1, kVecThreads, 0, st>>>(rowval, ptr, rows, n_sets, out, total);
  return cudaGetLastError();
}
cudaError_t launch_ds_update1(int rows, int nx, const int* set_of_row, float2* x, float2* r, const float2* p,
                              const float2* q, const double* rr, const double* pap, double* rowval, int* status,
                              cudaStream_t st) {
  note_launches(1); k_ds_update1<<<rows, kVecThreads, 0, st>>>(nx, set_of_row, x, r, p, q, rr, pap, rowval, status);
  return cudaGetLastError();
}
cudaError_t launch_ds_update2(int rows, int nx, const int* set_of_row, float2* p, const float2* r, const double* rr,
                              const double* rr_new, cudaStream_t st) {
  note_launches(1); k_ds_update2<<<rows, kVecThreads, 0, st>>>(nx, set_of_row, p, r, rr, rr_new);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FISTA --
// One block per 2^J x 2^J tile (J <= 5).  Per element:
//   z  = y - (N y - b + lam_tv grad TV_eps(y)) / L   (TV term of Eq. 17 when
//        lam_tv > 0; its gradient is computed beforehand by k_tv_grad)
//   x' = W^H soft_{lam/L}(W z)       (details only; tile-local Haar)
//   y' = x' + ck (x' - x),  x <- x'
__device__ __forceinline__ void haar_level_fwd(float2* t, float2* tmp, int ts, int h) {
  const float s = 0.70710678118654752440f;
  // along x on rows r < h, columns < h
  for (int i = threadIdx.x; i < h * (h / 2); i += blockDim.x) {
    const int r = i / (h / 2), c = i - r * (h / 2);
    const float2 a = t[r * ts + 2 * c], b = t[r * ts + 2 * c + 1];
    tmp[r * ts + c] = cscale(cadd(a, b), s);
    tmp[r * ts + h / 2 + c] = cscale(csub(a, b), s);
  }
  __syncthreads();
  // along y on columns < h
  for (int i = threadIdx.x; i < (h / 2) * h; i += blockDim.x) {
    const int r = i / h, c = i - r * h;
    const float2 a = tmp[(2 * r) * ts + c], b = tmp[(2 * r + 1) * ts + c];
    t[r * ts + c] = cscale(cadd(a, b), s);
    t[(h / 2 + r) * ts + c] = cscale(csub(a, b), s);
  }
  __syncthreads();
}

__device__ __forceinline__ void haar_level_inv(float2* t, float2* tmp, int ts, int h) {
  const float s = 0.70710678118654752440f;
  for (int i = threadIdx.x; i < (h / 2) * h; i += blockDim.x) {
    const int r = i / h, c = i - r * h;
    const float2 lo = t[r * ts + c], hi = t[(h / 2 + r) * ts + c];
    tmp[(2 * r) * ts + c] = cscale(cadd(lo, hi), s);
    tmp[(2 * r + 1) * ts + c] = cscale(csub(lo, hi), s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < h * (h / 2); i += blockDim.x) {
    const int r = i / (h / 2), c = i - r * (h / 2);
    const float2 lo = tmp[r * ts + c], hi = tmp[r * ts + h / 2 + c];
    t[r * ts + 2 * c] = cscale(cadd(lo, hi), s);
    t[r * ts + 2 * c + 1] = cscale(csub(lo, hi), s);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_fista_step(Geo g, const float2* __restrict__ parts, int nchunk,
                                                    float2* __restrict__ x, float2* __restrict__ y,
                                                    const float2* __restrict__ bvec, const double* Lip,
                                                    float lam, int levels, float ck,
                                                    const float2* __restrict__ tvg, float lam_tv, int* status) {
  __shared__ float2 t[32 * 33];
  __shared__ float2 tmp[32 * 33];
  const int ts = 1 << levels;
  const int tiles_x = g.nx / ts, tiles_y = g.ny / ts;
  const int tile = blockIdx.x;
  const int tz = tile / (tiles_x * tiles_y);
  const int rem = tile - tz * tiles_x * tiles_y;
  const int ty = rem / tiles_x, tx = rem - ty * tiles_x;
  const size_t L = (size_t)g.rows * g.nx;
  const double Ld = *Lip;
  const float invL = (Ld > 0.0 && isfinite(Ld)) ? (float)(1.0 / Ld) : 0.0f;
  if (!(Ld > 0.0 && isfinite(Ld)) && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(status, (int)kDevNonFinite);
  const float thr = lam * invL;
  for (int i = threadIdx.x; i < ts * ts; i += blockDim.x) {
    const int r = i / ts, c = i - r * ts;
    const size_t idx = ((size_t)tz * g.ny + ty * ts + r) * g.nx + tx * ts + c;
    float2 ny_ = parts[idx];
    for (int ch = 1; ch < nchunk; ++ch) ny_ = cadd(ny_, parts[ch * L + idx]);
    const float2 yv = y[idx], bv = bvec[idx];
    // gradient of the data term, plus lam_tv times the smoothed-TV gradient of y
    float2 gr = make_float2(ny_.x - bv.x, ny_.y - bv.y);
    if (tvg) {
      const float2 tv = tvg[idx];
      gr.x = fmaf(lam_tv, tv.x, gr.x);
      gr.y = fmaf(lam_tv, tv.y, gr.y);
    }
    t[r * 33 + c] = make_float2(yv.x - gr.x * invL, yv.y - gr.y * invL);
  }
  __syncthreads();
  for (int lev = 0, h = ts; lev < levels; ++lev, h >>= 1) haar_level_fwd(t, tmp, 33, h);
  for (int i = threadIdx.x; i < ts * ts; i += blockDim.x) {
    if (i == 0) continue;  // the coarsest approximation coefficient is not thresholded
    const int r = i / ts, c = i - r * ts;
    const float2 z = t[r * 33 + c];
    const float m = sqrtf(z.x * z.x + z.y * z.y);
    const float sc = m > thr ? 1.0f - thr / m : 0.0f;
    t[r * 33 + c] = cscale(z, sc);
  }
  __syncthreads();
  for (int lev = levels - 1; lev >= 0; --lev) haar_level_inv(t, tmp, 33, ts >> lev);
  for (int i = threadIdx.x; i < ts * ts; i += blockDim.x) {
    const int r = i / ts, c = i - r * ts;
    const size_t idx = ((size_t)tz * g.ny + ty * ts + r) * g.nx + tx * ts + c;
    const float2 xn = t[r * 33 + c];
    const float2 xo = x[idx];
    x[idx] = xn;
    y[idx] = make_float2(xn.x + ck * (xn.x - xo.x), xn.y + ck * (xn.y - xo.y));
  }
}

cudaError_t launch_fista_step(const Geo& g, const float2* parts, int nchunk, float2* x, float2* y,
                              const float2* b, const double* Lip, double lam, int levels, double ck,
                              const float2* tvg, double lam_tv, int* status, cudaStream_t st) {
  const int ts = 1 << levels;
  const int ntiles = (g.nx / ts) * (g.ny / ts) * g.nz;
  note_launches(1); k_fista_step<<<ntiles, 256, 0, st>>>(g, parts, nchunk, x, y, b, Lip, (float)lam, levels, (float)ck,
                                                          tvg, (float)lam_tv, status);
  return cudaGetLastError();
}

__global__ void k_add_scalar(double* d, double v) { d[0] += v; }
cudaError_t launch_add_scalar(double* d, double v, cudaStream_t st) {
  note_launches(1); k_add_scalar<<<1, 1, 0, st>>>(d, v);
  return cudaGetLastError();
}

}  // namespace gpjc
