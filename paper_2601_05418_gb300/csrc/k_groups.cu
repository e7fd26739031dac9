// Group construction (Sec. 2.4, Eq. 6-12) and patch compression (Eq. 13).
//
//  * plan tables: FFT twiddles, readout pre-twiddles and the wave excursion
//    a_y(t), a_z(t) of Eq. 3, computed in double on the device;
//  * ROI compaction (raster order) and whitened, pixel-normalised coil
//    values c^_n(r) = (T c)_n(r) / sqrt(w sum_n |(T c)_n(r)|^2);
//  * Gram P_g = sum_r v_r v_r^H (Eq. 9-11) with v_r[(n,tau)] =
//    c^_n(r) exp(-i [2 pi t_c x_c / N_tx + phi(t,y,z)]), t = p_g w + tau:
//    FP32 products and FP32 sums over 256-pixel runs, FP64 across runs and
//    across pixel slabs (FP64 atomics into P);
//  * eigen-decomposition of P_g (Eq. 8) for the leading N_s' vectors:
//    FP64 block subspace iteration with classical Gram-Schmidt applied twice,
//    then Rayleigh-Ritz with a parallel-ordered complex Jacobi solver;
//  * A_g = C_g U_g^H (T (x) I_w) (Eq. 12), stored row-major and transposed;
//  * S'_{l,p} = A_{g(p)} s_{l,p} (Eq. 13) in FP32.
#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

// ------------------------------------------------------------------ tables --
// Twiddle table of one FFT length n: exp(-2 pi i e / n) at position k, with
// e = k for the radix-stage plan and e = (k mod n2) (k / n2) for the two-pass
// plan n = n1 n2 (position k1 n2 + i2 holds the twiddle of i2 k1).
__device__ __forceinline__ float2 fft_twiddle(int k, int n, int n2) {
  const int e = n2 > 0 ? (k % n2) * (k / n2) : k;
  double s, c;
  sincospi(-2.0 * (double)e / n, &s, &c);
  return make_float2((float)c, (float)s);
}

__global__ void k_make_tables(int nx, int ny, int nz, int os, int n2x, int n2y, int n2z, float2* tw_x,
                              float2* tw_y, float2* tw_z, float2* pre, float* ay, float* az, double cycles,
                              double kappa_y, double kappa_z) {
  const int ntx = os * nx;
  const int total = nx + ny + nz + ntx + ntx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    double s, c;
    int k = i;
    if (k < nx) {
      tw_x[k] = fft_twiddle(k, nx, n2x);
      continue;
    }
    k -= nx;
    if (k < ny) {
      tw_y[k] = fft_twiddle(k, ny, n2y);
      continue;
    }
    k -= ny;
    if (k < nz) {
      tw_z[k] = fft_twiddle(k, nz, n2z);
      continue;
    }
    k -= nz;
    if (k < ntx) {
      const int sh = k / nx, x = k - sh * nx;
      // (-1)^x exp(-2 pi i s x / ntx); s x < ntx * nx, reduce modulo ntx exactly
      const long long e = ((long long)sh * x) % ntx;
      sincospi(-2.0 * (double)e / ntx, &s, &c);
      const float sg = (x & 1) ? -1.0f : 1.0f;
      pre[k] = make_float2(sg * (float)c, sg * (float)s);
      continue;
    }
    k -= ntx;
    // theta = 2 pi cycles t / ntx
    const double th = 2.0 * cycles * k / ntx;  // in units of pi
    sincospi(th, &s, &c);
    ay[k] = (float)(kappa_y * (1.0 - c) * 0.5);
    az[k] = (float)(kappa_z * s * 0.5);
  }
}

cudaError_t launch_make_tables(Geo& g, float2* tw_x, float2* tw_y, float2* tw_z, float2* pre, float* ay,
                               float* az, double cycles, double kappa_y, double kappa_z, cudaStream_t st) {
  const int total = g.nx + g.ny + g.nz + 2 * g.ntx;
  note_launches(1); k_make_tables<<<(total + 255) / 256, 256, 0, st>>>(g.nx, g.ny, g.nz, g.os, g.fx.n2, g.fy.n2,
                                                                      g.fz.n2, tw_x, tw_y, tw_z, pre, ay, az,
                                                                      cycles, kappa_y, kappa_z);
  return cudaGetLastError();
}

// post_y[y][t] = (-1)^{m + nx/2} e^{i pi s/os} e^{-2 pi i a_y(t) y_c/ny} / sqrt(ntx)
// post_z[z][t] = e^{-2 pi i a_z(t) z_c/nz}, t = os m + s (double precision).
__global__ void k_make_post(int nx, int ny, int nz, int os, float2* post_y, float2* post_z, double cycles,
                            double kappa_y, double kappa_z) {
  const int ntx = os * nx;
  const size_t ny_tot = (size_t)ny * ntx, total = ny_tot + (size_t)nz * ntx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const bool isy = i < ny_tot;
    const size_t j = isy ? i : i - ny_tot;
    const int r = (int)(j / ntx), t = (int)(j - (size_t)r * ntx);
    double s, c;
    sincospi(2.0 * cycles * t / ntx, &s, &c);
    double arg;  // in units of pi
    float scale = 1.0f;
    if (isy) {
      const int m = t / os, sh = t - m * os;
      const double ay = kappa_y * (1.0 - c) * 0.5;
      arg = (double)sh / os - 2.0 * ay * (double)(r - ny / 2) / ny;
      scale = (float)((((m + nx / 2) & 1) ? -1.0 : 1.0) / sqrt((double)ntx));
    } else {
      const double az = kappa_z * s * 0.5;
      arg = nz > 1 ? -2.0 * az * (double)(r - nz / 2) / nz : 0.0;
    }
    double ps, pc;
    sincospi(arg, &ps, &pc);
    float2 v = make_float2((float)pc * scale, (float)ps * scale);
    if (isy)
      post_y[j] = v;
    else
      post_z[j] = v;
  }
}

cudaError_t launch_make_post(const Geo& g, float2* post_y, float2* post_z, double cycles, double kappa_y,
                             double kappa_z, cudaStream_t st) {
  note_launches(1); k_make_post<<<1024, 256, 0, st>>>(g.nx, g.ny, g.nz, g.os, post_y, post_z, cycles, kappa_y,
                                                      kappa_z);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ ROI --
constexpr int kRoiThreads = 256;
constexpr int kRoiPer = 4;  // pixels per thread per block
int roi_block_pixels() { return kRoiThreads * kRoiPer; }

__device__ __forceinline__ bool roi_valid(const Geo& g, const float2* coil, const uint8_t* roi, size_t L,
                                          size_t i) {
  if (i >= L || !roi[i]) return false;
  float s = 0.f;
  for (int n = 0; n < g.nc; ++n) {
    float2 c = coil[n * L + i];
    s += c.x * c.x + c.y * c.y;
  }
  return s > 0.f;
}

__global__ void k_roi_count(Geo g, const float2* __restrict__ coil, const uint8_t* __restrict__ roi,
                            int* blockcount) {
  const size_t L = (size_t)g.rows * g.nx;
  int cnt = 0;
  for (int r = 0; r < kRoiPer; ++r) {
    const size_t i = (size_t)blockIdx.x * kRoiThreads * kRoiPer + r * kRoiThreads + threadIdx.x;
    cnt += roi_valid(g, coil, roi, L, i) ? 1 : 0;
  }
  __shared__ int sc[kRoiThreads / 32];
  int wsum = cnt;
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  if ((threadIdx.x & 31) == 0) sc[threadIdx.x >> 5] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kRoiThreads / 32; ++w) t += sc[w];
    blockcount[blockIdx.x] = t;
  }
}

__global__ void k_roi_scan(const int* blockcount, int* blockoff, int nblk, int* total) {
  __shared__ int buf[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nblk ? blockcount[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblk) blockoff[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_roi_compact(Geo g, const float2* __restrict__ coil, const uint8_t* __restrict__ roi,
                              const int* __restrict__ blockoff, int* __restrict__ pix) {
  const size_t L = (size_t)g.rows * g.nx;
  __shared__ int wcount[kRoiThreads / 32];
  __shared__ int running;
  if (threadIdx.x == 0) running = blockoff[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = 0; r < kRoiPer; ++r) {
    const size_t i = (size_t)blockIdx.x * kRoiThreads * kRoiPer + r * kRoiThreads + threadIdx.x;
    const bool v = roi_valid(g, coil, roi, L, i);
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    if (lane == 0) wcount[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wcount[w];
    const int pos = running + before + __popc(bal & ((1u << lane) - 1u));
    if (v) pix[pos] = (int)i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < kRoiThreads / 32; ++w) t += wcount[w];
      running += t;
    }
    __syncthreads();
  }
}

// chat[n][k] = (T c)_n(r_k) / sqrt(w * sum_n |(T c)_n(r_k)|^2); zero for k >= K.
// K = |ROI| is read on the device; rows of chat are `Kpad` apart (>= the
// padded K), entries in [K, round_up(K, 32)) are zero.
__global__ void k_roi_coils(Geo g, const float2* __restrict__ coil, const float2* __restrict__ T,
                            const int* __restrict__ pix, const int* __restrict__ dK, int Kpad,
                            float2* __restrict__ chat) {
  const size_t L = (size_t)g.rows * g.nx;
  const int K = *dK;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ((K + 31) / 32) * 32) return;
  if (k >= K) {
    for (int n = 0; n < g.nc; ++n) chat[(size_t)n * Kpad + k] = make_float2(0.f, 0.f);
    return;
  }
  const size_t r = (size_t)pix[k];
  double s = 0.0;
  if (T == nullptr) {
    for (int n = 0; n < g.nc; ++n) {
      float2 c = coil[n * L + r];
      s += (double)c.x * c.x + (double)c.y * c.y;
    }
    const float inv = (float)(1.0 / sqrt((double)g.w * s));
    for (int n = 0; n < g.nc; ++n) chat[(size_t)n * Kpad + k] = cscale(coil[n * L + r], inv);
    return;
  }
  // whitened: (T c)_n = sum_m T[n][m] c_m; computed twice to avoid a large
  // per-thread array (nc is at most 64).
  for (int n = 0; n < g.nc; ++n) {
    double re = 0.0, im = 0.0;
    for (int m = 0; m < g.nc; ++m) {
      const float2 t = T[n * g.nc + m];
      const float2 c = coil[m * L + r];
      re += (double)t.x * c.x - (double)t.y * c.y;
      im += (double)t.x * c.y + (double)t.y * c.x;
    }
    s += re * re + im * im;
  }
  const double inv = 1.0 / sqrt((double)g.w * s);
  for (int n = 0; n < g.nc; ++n) {
    double re = 0.0, im = 0.0;
    for (int m = 0; m < g.nc; ++m) {
      const float2 t = T[n * g.nc + m];
      const float2 c = coil[m * L + r];
      re += (double)t.x * c.x - (double)t.y * c.y;
      im += (double)t.x * c.y + (double)t.y * c.x;
    }
    chat[(size_t)n * Kpad + k] = make_float2((float)(re * inv), (float)(im * inv));
  }
}

cudaError_t launch_roi_count(const Geo& g, const float2* coil, const uint8_t* roi, int* blockcount, int nblk,
                             cudaStream_t st) {
  note_launches(1); k_roi_count<<<nblk, kRoiThreads, 0, st>>>(g, coil, roi, blockcount);
  return cudaGetLastError();
}
cudaError_t launch_roi_scan(const int* blockcount, int* blockoff, int nblk, int* total, cudaStream_t st) {
  note_launches(1); k_roi_scan<<<1, 1024, 0, st>>>(blockcount, blockoff, nblk, total);
  return cudaGetLastError();
}
cudaError_t launch_roi_compact(const Geo& g, const float2* coil, const uint8_t* roi, const int* blockoff,
                               int* pix, int nblk, cudaStream_t st) {
  note_launches(1); k_roi_compact<<<nblk, kRoiThreads, 0, st>>>(g, coil, roi, blockoff, pix);
  return cudaGetLastError();
}
cudaError_t launch_roi_coils(const Geo& g, const float2* coil, const float2* T, const int* pix, const int* dK,
                             int Kpad, float2* chat, cudaStream_t st) {
  note_launches(1); k_roi_coils<<<(Kpad + 255) / 256, 256, 0, st>>>(g, coil, T, pix, dK, Kpad, chat);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Gram --
constexpr int kGT = 64;        // Gram tile (rows and columns of P)
constexpr int kGKC = 32;       // pixels per chunk
constexpr int kGFlush = 8;     // chunks per FP32 run (256 pixels)
constexpr int kGSlab = 2048;   // pixels per block (FP64 atomics across slabs)

__global__ void __launch_bounds__(256) k_gram(Geo g, const float2* __restrict__ chat,
                                              const int* __restrict__ pix, const int* __restrict__ dK,
                                              int Kpad, const int* __restrict__ pref,
                                              double2* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  double2* acc64 = (double2*)gsm_raw;              // [kGT * kGT] FP64 sums, thread-owned slots
  float2* As = (float2*)(acc64 + kGT * kGT);      // [kGKC][kGT]
  float2* Bs = As + kGKC * kGT;                   // [kGKC][kGT]
  float2* psi = Bs + kGKC * kGT;                  // [w][kGKC]
  const int grp = blockIdx.y;
  // tile pair (I <= J) from the linear index
  const int nt = (g.ns + kGT - 1) / kGT;
  int pidx = blockIdx.x, I = 0;
  while (pidx >= nt - I) {
    pidx -= nt - I;
    ++I;
  }
  const int J = I + pidx;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int t0 = pref[grp] * g.w;
  const int K = *dK;
  const int k_begin = blockIdx.z * kGSlab;
  const int k_end = min(((K + kGKC - 1) / kGKC) * kGKC, k_begin + kGSlab);
  if (k_begin >= k_end) return;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc64[(ty * 4 + a) * kGT + tx * 4 + b] = make_double2(0.0, 0.0);
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  int run = 0;
  const float inv_ny = 1.0f / (float)g.ny;
  const float inv_nz = 1.0f / (float)g.nz;
  for (int k0 = k_begin; k0 < k_end; k0 += kGKC) {
    // phases psi[tau][r]
    for (int i = threadIdx.x; i < g.w * kGKC; i += blockDim.x) {
      const int tau = i / kGKC, r = i - tau * kGKC;
      const int k = k0 + r;
      float2 e = make_float2(0.f, 0.f);
      if (k < K) {
        const int p = pix[k];
        const int x = p % g.nx;
        const int row = p / g.nx;
        const int y = row % g.ny, z = row / g.ny;
        const int t = t0 + tau;
        int prod = ((t - g.ntx / 2) * (x - g.nx / 2)) % g.ntx;
        if (prod < 0) prod += g.ntx;
        const float wave = g.ay[t] * (float)(y - g.ny / 2) * inv_ny +
                           (g.nz > 1 ? g.az[t] * (float)(z - g.nz / 2) * inv_nz : 0.0f);
        const float arg = -(2.0f * (float)prod / (float)g.ntx + 2.0f * wave);
        e = expipi(arg);
      }
      psi[i] = e;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kGKC * kGT; i += blockDim.x) {
      const int r = i / kGT, ii = i - r * kGT;
      const int ra = I * kGT + ii, rb = J * kGT + ii;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (ra < g.ns) {
        const int n = ra / g.w, tau = ra - n * g.w;
        va = cmul(chat[(size_t)n * Kpad + k0 + r], psi[tau * kGKC + r]);
      }
      if (rb < g.ns) {
        const int n = rb / g.w, tau = rb - n * g.w;
        vb = cmul(chat[(size_t)n * Kpad + k0 + r], psi[tau * kGKC + r]);
      }
      As[i] = va;
      Bs[i] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kGKC; ++r) {
      float2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[r * kGT + ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[r * kGT + tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfmac(acc[a][b], bv[b], av[a]);  // a * conj(b)
    }
    __syncthreads();
    if (++run == kGFlush || k0 + kGKC >= k_end) {
      run = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          double2& d = acc64[(ty * 4 + a) * kGT + tx * 4 + b];
          d.x += acc[a][b].x;
          d.y += acc[a][b].y;
          acc[a][b] = make_float2(0.f, 0.f);
        }
    }
  }
  double2* Pg = P + (size_t)grp * g.ns * g.ns;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = I * kGT + ty * 4 + a, j = J * kGT + tx * 4 + b;
      if (i < g.ns && j < g.ns && i <= j) {
        const double2 v = acc64[(ty * 4 + a) * kGT + tx * 4 + b];
        double2* d = Pg + (size_t)i * g.ns + j;
        atomicAdd(&d->x, v.x);
        atomicAdd(&d->y, v.y);
      }
    }
}

// P[i][j] = conj(P[j][i]) for i > j; real diagonal.
__global__ void k_hermitize(int ns, double2* P) {
  double2* Pg = P + (size_t)blockIdx.y * ns * ns;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ns * ns; idx += gridDim.x * blockDim.x) {
    const int i = idx / ns, j = idx - i * ns;
    if (i > j) {
      const double2 u = Pg[(size_t)j * ns + i];
      Pg[idx] = make_double2(u.x, -u.y);
    } else if (i == j) {
      Pg[idx].y = 0.0;
    }
  }
}

cudaError_t launch_gram(const Geo& g, const float2* chat, const int* pix, const int* dK, int Kpad,
                        const int* pref, double2* P, cudaStream_t st) {
  const int nt = (g.ns + kGT - 1) / kGT;
  const int npairs = nt * (nt + 1) / 2;
  const int nslab = (Kpad + kGSlab - 1) / kGSlab;
  const size_t sm = sizeof(double2) * (size_t)kGT * kGT + sizeof(float2) * (size_t)(2 * kGKC * kGT + g.w * kGKC);
  cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_gram, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  note_launches(1); k_gram<<<dim3(npairs, g.G, nslab), 256, sm, st>>>(g, chat, pix, dK, Kpad, pref, P);
  return cudaGetLastError();
}

cudaError_t launch_hermitize(const Geo& g, double2* P, cudaStream_t st) {
  const int nb = (g.ns * g.ns + 255) / 256;
  note_launches(1); k_hermitize<<<dim3(nb < 1024 ? nb : 1024, g.G), 256, 0, st>>>(g.ns, P);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ eig --
// Complex FP64 helpers.
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ void zfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void zfmac(double2& acc, double2 a, double2 b) {  // += conj(a) b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ double hash_unit(unsigned long long v) {
  // splitmix64 -> [-1, 1)
  v += 0x9E3779B97F4A7C15ull;
  v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
  v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
  v ^= v >> 31;
  return (double)(v >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void k_eig_init(int ns, int b, double2* X) {
  const size_t n = (size_t)ns * b;
  double2* Xg = X + blockIdx.y * n;
  for (size_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long key = ((unsigned long long)blockIdx.y << 40) ^ (i << 1);
    Xg[i] = make_double2(hash_unit(key), hash_unit(key | 1ull));
  }
}

cudaError_t launch_eig_init(const Geo& g, int b, double2* X, cudaStream_t st) {
  note_launches(1); k_eig_init<<<dim3(64, g.G), 256, 0, st>>>(g.ns, b, X);
  return cudaGetLastError();
}

// Y[g] = P[g] X[g]; P is ns x ns, X is ns x b (row-major), b <= kEigMaxB.
constexpr int kEigMaxB = 96;
constexpr int kMMRows = 32, kMMK = 32;
__global__ void __launch_bounds__(256) k_eig_matmul(int ns, int b, const double2* __restrict__ P,
                                                    const double2* __restrict__ X, double2* __restrict__ Y) {
  __shared__ double2 Ps[kMMRows][kMMK + 1];
  extern __shared__ double2 Xs[];  // [kMMK][b]
  const int grp = blockIdx.y;
  const double2* Pg = P + (size_t)grp * ns * ns;
  const double2* Xg = X + (size_t)grp * ns * b;
  double2* Yg = Y + (size_t)grp * ns * b;
  const int r0 = blockIdx.x * kMMRows;
  constexpr int MAXO = kMMRows * kEigMaxB / 256;  // 12
  double2 acc[MAXO];
#pragma unroll
  for (int j = 0; j < MAXO; ++j) acc[j] = make_double2(0.0, 0.0);
  const int nout = kMMRows * b;
  for (int k0 = 0; k0 < ns; k0 += kMMK) {
    for (int i = threadIdx.x; i < kMMRows * kMMK; i += blockDim.x) {
      const int r = i / kMMK, kk = i - r * kMMK;
      const int gr = r0 + r, gk = k0 + kk;
      Ps[r][kk] = (gr < ns && gk < ns) ? Pg[(size_t)gr * ns + gk] : make_double2(0.0, 0.0);
    }
    for (int i = threadIdx.x; i < kMMK * b; i += blockDim.x) {
      const int kk = i / b, c = i - kk * b;
      const int gk = k0 + kk;
      Xs[i] = gk < ns ? Xg[(size_t)gk * b + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MAXO; ++j) {
      const int o = threadIdx.x + j * 256;
      if (o < nout) {
        const int r = o / b, c = o - r * b;
        double2 a = acc[j];
        for (int kk = 0; kk < kMMK; ++kk) zfma(a, Ps[r][kk], Xs[kk * b + c]);
        acc[j] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < MAXO; ++j) {
    const int o = threadIdx.x + j * 256;
    if (o < nout) {
      const int r = o / b, c = o - r * b;
      if (r0 + r < ns) Yg[(size_t)(r0 + r) * b + c] = acc[j];
    }
  }
}

cudaError_t launch_eig_matmul(const Geo& g, int b, const double2* P, const double2* X, double2* Y,
                              cudaStream_t st) {
  if (b > kEigMaxB) return cudaErrorInvalidValue;
  const size_t sm = sizeof(double2) * (size_t)kMMK * b;
  cudaFuncSetAttribute(k_eig_matmul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k_eig_matmul<<<dim3((g.ns + kMMRows - 1) / kMMRows, g.G), 256, sm, st>>>(g.ns, b, P, X, Y);
  return cudaGetLastError();
}

// ---- FP32 phase of the subspace iteration (same algorithm in single
// precision; the FP64 iterations that follow refine its subspace)
__global__ void k_to_f32(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_to_f64(const float2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = make_double2((double)a[i].x, (double)a[i].y);
}
cudaError_t launch_to_f32(const double2* a, float2* b, size_t n, cudaStream_t st) {
  note_launches(1); k_to_f32<<<1024, 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}
cudaError_t launch_to_f64(const float2* a, double2* b, size_t n, cudaStream_t st) {
  note_launches(1); k_to_f64<<<1024, 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_eig_matmul32(int ns, int b, const float2* __restrict__ P,
                                                      const float2* __restrict__ X, float2* __restrict__ Y) {
  __shared__ float2 Ps[kMMRows][kMMK + 1];
  extern __shared__ float2 Xs32[];  // [kMMK][b]
  const int grp = blockIdx.y;
  const float2* Pg = P + (size_t)grp * ns * ns;
  const float2* Xg = X + (size_t)grp * ns * b;
  float2* Yg = Y + (size_t)grp * ns * b;
  const int r0 = blockIdx.x * kMMRows;
  constexpr int MAXO = kMMRows * kEigMaxB / 256;
  float2 acc[MAXO];
#pragma unroll
  for (int j = 0; j < MAXO; ++j) acc[j] = make_float2(0.f, 0.f);
  const int nout = kMMRows * b;
  for (int k0 = 0; k0 < ns; k0 += kMMK) {
    for (int i = threadIdx.x; i < kMMRows * kMMK; i += blockDim.x) {
      const int r = i / kMMK, kk = i - r * kMMK;
      const int gr = r0 + r, gk = k0 + kk;
      Ps[r][kk] = (gr < ns && gk < ns) ? Pg[(size_t)gr * ns + gk] : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < kMMK * b; i += blockDim.x) {
      const int kk = i / b, c = i - kk * b;
      const int gk = k0 + kk;
      Xs32[i] = gk < ns ? Xg[(size_t)gk * b + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MAXO; ++j) {
      const int o = threadIdx.x + j * 256;
      if (o < nout) {
        const int r = o / b, c = o - r * b;
        float2 a = acc[j];
        for (int kk = 0; kk < kMMK; ++kk) cfma(a, Ps[r][kk], Xs32[kk * b + c]);
        acc[j] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < MAXO; ++j) {
    const int o = threadIdx.x + j * 256;
    if (o < nout) {
      const int r = o / b, c = o - r * b;
      if (r0 + r < ns) Yg[(size_t)(r0 + r) * b + c] = acc[j];
    }
  }
}

cudaError_t launch_eig_matmul32(const Geo& g, int b, const float2* P, const float2* X, float2* Y, cudaStream_t st) {
  if (b > kEigMaxB) return cudaErrorInvalidValue;
  const size_t sm = sizeof(float2) * (size_t)kMMK * b;
  cudaFuncSetAttribute(k_eig_matmul32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k_eig_matmul32<<<dim3((g.ns + kMMRows - 1) / kMMRows, g.G), 256, sm, st>>>(g.ns, b, P, X, Y);
  return cudaGetLastError();
}

// Orthonormalise the columns of Y[g] (ns x b, row-major) in place: classical
// Gram-Schmidt with one re-orthogonalisation pass per column (CGS2), a
// column that vanishes is replaced by a unit vector.  One block per group;
// when the group's block fits in shared memory (SM) all passes run there.
// C is float2 (FP32 phase) or double2; norms are accumulated in double.
__device__ __forceinline__ void cacc_conj(float2& s, float2 a, float2 b) { cfmac(s, a, b); }
__device__ __forceinline__ void cacc_conj(double2& s, double2 a, double2 b) { zfmac(s, a, b); }
__device__ __forceinline__ float2 cmk(double re, double im, float2*) { return make_float2((float)re, (float)im); }
__device__ __forceinline__ double2 cmk(double re, double im, double2*) { return make_double2(re, im); }
__device__ __forceinline__ float wsum(float v) { return warp_sumf(v); }
__device__ __forceinline__ double wsum(double v) { return warp_sum(v); }

template <typename C, bool SM>
__global__ void __launch_bounds__(256) k_eig_orth_t(int ns, int b, C* Y) {
  extern __shared__ __align__(16) unsigned char orth_sm[];
  C* v = (C*)orth_sm;  // [ns]
  C* h = v + ns;       // [b]
  C* Ys = h + b;       // [ns][b + 1] when SM (odd row stride: no bank conflicts down a column)
  __shared__ double red[32];
  __shared__ double nrm;
  C* Yg = Y + (size_t)blockIdx.x * ns * b;
  C* Yw = SM ? Ys : Yg;
  const int ld = SM ? b + 1 : b;
  if (SM) {
    for (int i = threadIdx.x; i < ns * b; i += blockDim.x) Ys[(i / b) * ld + i % b] = Yg[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < b; ++c) {
    for (int attempt = 0; attempt < 2; ++attempt) {
      for (int i = threadIdx.x; i < ns; i += blockDim.x)
        v[i] = attempt == 0 ? Yw[(size_t)i * ld + c] : cmk(i == (c % ns) ? 1.0 : 0.0, 0.0, (C*)nullptr);
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        // h_j = <y_j, v> for the c finished columns (one warp per column)
        for (int j = wid; j < c; j += nw) {
          C sacc = cmk(0.0, 0.0, (C*)nullptr);
          for (int i = lane; i < ns; i += 32) cacc_conj(sacc, Yw[(size_t)i * ld + j], v[i]);
          sacc.x = wsum(sacc.x);
          sacc.y = wsum(sacc.y);
          if (lane == 0) h[j] = sacc;
        }
        __syncthreads();
        // v -= Y_{<c} h
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
          C a = v[i];
          const C* yr = Yw + (size_t)i * ld;
          for (int j = 0; j < c; ++j) {
            const C q = yr[j], hj = h[j];
            a.x -= q.x * hj.x - q.y * hj.y;
            a.y -= q.x * hj.y + q.y * hj.x;
          }
          v[i] = a;
        }
        __syncthreads();
      }
      double sq = 0.0;
      for (int i = threadIdx.x; i < ns; i += blockDim.x) sq += (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
      sq = block_sum(sq, red);
      if (threadIdx.x == 0) nrm = sqrt(sq);
      __syncthreads();
      const double nv = nrm;
      if (nv > (sizeof(C) == sizeof(float2) ? 1e-30 : 1e-280)) {
        const double inv = 1.0 / nv;
        for (int i = threadIdx.x; i < ns; i += blockDim.x)
          Yw[(size_t)i * ld + c] = cmk(v[i].x * inv, v[i].y * inv, (C*)nullptr);
        __syncthreads();
        break;
      }
      __syncthreads();
    }
  }
  if (SM) {
    for (int i = threadIdx.x; i < ns * b; i += blockDim.x) Yg[i] = Ys[(i / b) * ld + i % b];
  }
}

template <typename C>
static cudaError_t launch_orth_t(const Geo& g, int b, C* Y, cudaStream_t st) {
  const size_t base = sizeof(C) * (size_t)(g.ns + b);
  const size_t full = base + sizeof(C) * (size_t)g.ns * (b + 1);
  if (full <= 200 * 1024) {
    cudaFuncSetAttribute(k_eig_orth_t<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)full);
    note_launches(1); k_eig_orth_t<C, true><<<g.G, 256, full, st>>>(g.ns, b, Y);
  } else {
    cudaFuncSetAttribute(k_eig_orth_t<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
    note_launches(1); k_eig_orth_t<C, false><<<g.G, 256, base, st>>>(g.ns, b, Y);
  }
  return cudaGetLastError();
}

cudaError_t launch_eig_orth32(const Geo& g, int b, float2* Y, cudaStream_t st) { return launch_orth_t(g, b, Y, st); }
cudaError_t launch_eig_orth(const Geo& g, int b, double2* Y, cudaStream_t st) { return launch_orth_t(g, b, Y, st); }

// Hm[g][a][c] = sum_i conj(Q[i][a]) Z[i][c]
__global__ void k_eig_project(int ns, int b, const double2* __restrict__ Q, const double2* __restrict__ Z,
                              double2* __restrict__ Hm) {
  const int grp = blockIdx.y;
  const double2* Qg = Q + (size_t)grp * ns * b;
  const double2* Zg = Z + (size_t)grp * ns * b;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= b * b) return;
  const int a = o / b, c = o - a * b;
  double2 s = make_double2(0.0, 0.0);
  for (int i = 0; i < ns; ++i) zfmac(s, Qg[(size_t)i * b + a], Zg[(size_t)i * b + c]);
  Hm[(size_t)grp * b * b + o] = s;
}

cudaError_t launch_eig_project(const Geo& g, int b, const double2* Q, const double2* Z, double2* Hm,
                               cudaStream_t st) {
  note_launches(1); k_eig_project<<<dim3((b * b + 127) / 128, g.G), 128, 0, st>>>(g.ns, b, Q, Z, Hm);
  return cudaGetLastError();
}

// Parallel-ordered (round-robin) two-sided complex Jacobi on the b x b
// Hermitian Rayleigh quotient Hm[g]; W[g] accumulates the rotations.
// ritz[g][c] = eigenvalues, order[g][r] = index of the r-th largest
// (descending, ties by index).
__global__ void __launch_bounds__(256) k_eig_jacobi(int b, double2* __restrict__ Hm, double2* __restrict__ W,
                                                    double* __restrict__ ritz, int* __restrict__ order,
                                                    int max_sweeps, int wsm) {
  extern __shared__ double2 jsm[];
  const int n = b + (b & 1);  // even player count (a dummy when b is odd)
  double2* H = jsm;           // [b][b]
  const int grp_ = blockIdx.x;
  // rotations accumulate in shared memory when H and W fit there together
  // (written to W at the end), else directly in W
  double2* Ws = wsm ? jsm + b * b : W + (size_t)grp_ * b * b;
  __shared__ int perm[kEigMaxB + 2];
  __shared__ int pp[kEigMaxB / 2 + 1], pq[kEigMaxB / 2 + 1];
  __shared__ double pc[kEigMaxB / 2 + 1], ps[kEigMaxB / 2 + 1];
  __shared__ double2 pe[kEigMaxB / 2 + 1];
  __shared__ double red[32];
  __shared__ int done;
  const int grp = blockIdx.x;
  double2* Hg = Hm + (size_t)grp * b * b;
  double2* Wg = W + (size_t)grp * b * b;
  for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
    double2 v = Hg[i];
    const int r = i / b, c = i - r * b;
    if (r > c) {  // use the upper triangle as the master copy
      const double2 u = Hg[(size_t)c * b + r];
      v = make_double2(u.x, -u.y);
    } else if (r == c) {
      v.y = 0.0;
    }
    H[i] = v;
    Ws[i] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test on the off-diagonal mass
    double off = 0.0, dia = 0.0;
    for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
      const int r = i / b, c = i - r * b;
      const double m = H[i].x * H[i].x + H[i].y * H[i].y;
      if (r == c)
        dia += m;
      else
        off += m;
    }
    off = block_sum(off, red);
    __syncthreads();
    dia = block_sum(dia, red);
    if (threadIdx.x == 0) done = (off <= 1e-30 * dia) ? 1 : 0;
    __syncthreads();
    if (done) break;
    for (int step = 0; step < n - 1; ++step) {
      const int half = n / 2;
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p = perm[k], q = perm[n - 1 - k];
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        pp[k] = p;
        pq[k] = q;
        double c = 1.0, s = 0.0;
        double2 e = make_double2(1.0, 0.0);
        if (q < b) {
          const double2 h = H[p * b + q];
          const double ah = hypot(h.x, h.y);
          const double a = H[p * b + p].x, d = H[q * b + q].x;
          if (ah > 1e-300 && ah > 1e-18 * (fabs(a) + fabs(d))) {
            const double zeta = (d - a) / (2.0 * ah);
            const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            e = make_double2(h.x / ah, h.y / ah);
          }
        }
        pc[k] = c;
        ps[k] = s;
        pe[k] = e;
      }
      __syncthreads();
      // rows: G^H from the left
      for (int i = threadIdx.x; i < half * b; i += blockDim.x) {
        const int k = i / b, j = i - k * b;
        const int p = pp[k], q = pq[k];
        if (q >= b || ps[k] == 0.0) continue;
        const double c = pc[k], s = ps[k];
        const double2 e = pe[k];
        const double2 rp = H[p * b + j], rq = H[q * b + j];
        const double2 erq = zmul(e, rq);              // e^{i a} rq
        const double2 erp = zmulc(e, rp);             // e^{-i a} rp
        H[p * b + j] = zsub(zscale(rp, c), zscale(erq, s));
        H[q * b + j] = zadd(zscale(erp, s), zscale(rq, c));
      }
      __syncthreads();
      // columns: G from the right, also on W
      for (int i = threadIdx.x; i < half * b; i += blockDim.x) {
        const int k = i / b, r = i - k * b;
        const int p = pp[k], q = pq[k];
        if (q >= b || ps[k] == 0.0) continue;
        const double c = pc[k], s = ps[k];
        const double2 e = pe[k];
        double2 cp = H[r * b + p], cq = H[r * b + q];
        H[r * b + p] = zsub(zscale(cp, c), zscale(zmulc(e, cq), s));
        H[r * b + q] = zadd(zscale(zmul(e, cp), s), zscale(cq, c));
        cp = Ws[r * b + p];
        cq = Ws[r * b + q];
        Ws[r * b + p] = zsub(zscale(cp, c), zscale(zmulc(e, cq), s));
        Ws[r * b + q] = zadd(zscale(zmul(e, cp), s), zscale(cq, c));
      }
      __syncthreads();
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        const int p = pp[k], q = pq[k];
        if (q < b && ps[k] != 0.0) {
          H[p * b + q] = make_double2(0.0, 0.0);
          H[q * b + p] = make_double2(0.0, 0.0);
          H[p * b + p].y = 0.0;
          H[q * b + q].y = 0.0;
        }
      }
      __syncthreads();
      // round-robin rotation of players 1..n-1
      if (threadIdx.x == 0) {
        const int last = perm[n - 1];
        for (int i = n - 1; i > 1; --i) perm[i] = perm[i - 1];
        perm[1] = last;
      }
      __syncthreads();
    }
  }
  for (int c = threadIdx.x; c < b; c += blockDim.x) ritz[(size_t)grp * b + c] = H[c * b + c].x;
  if (wsm)
    for (int i = threadIdx.x; i < b * b; i += blockDim.x) Wg[i] = Ws[i];
  __syncthreads();
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    const double v = H[c * b + c].x;
    int rank = 0;
    for (int c2 = 0; c2 < b; ++c2) {
      const double v2 = H[c2 * b + c2].x;
      if (v2 > v || (v2 == v && c2 < c)) ++rank;
    }
    order[(size_t)grp * b + rank] = c;
  }
}

cudaError_t launch_eig_jacobi(const Geo& g, int b, double2* Hm, double2* W, double* ritz, int* order,
                              int max_sweeps, cudaStream_t st) {
  if (b > kEigMaxB) return cudaErrorInvalidValue;
  const int wsm = 2 * sizeof(double2) * (size_t)b * b <= (size_t)200 * 1024 ? 1 : 0;
  const size_t sm = (wsm ? 2 : 1) * sizeof(double2) * (size_t)b * b;
  cudaFuncSetAttribute(k_eig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launches(1); k_eig_jacobi<<<g.G, 256, sm, st>>>(b, Hm, W, ritz, order, max_sweeps, wsm);
  return cudaGetLastError();
}

// U[g][i][r] = sum_j Q[i][j] W[j][order[r]]  (Ritz vectors, descending)
__global__ void k_eig_rotate(int ns, int b, const double2* __restrict__ Q, const double2* __restrict__ W,
                             const int* __restrict__ order, double2* __restrict__ U) {
  const int grp = blockIdx.y;
  const size_t n = (size_t)ns * b;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(o / b), r = (int)(o - (size_t)i * b);
    const int col = order[(size_t)grp * b + r];
    const double2* Qi = Q + (size_t)grp * n + (size_t)i * b;
    const double2* Wg = W + (size_t)grp * b * b;
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < b; ++j) zfma(s, Qi[j], Wg[(size_t)j * b + col]);
    U[(size_t)grp * n + o] = s;
  }
}

cudaError_t launch_eig_rotate(const Geo& g, int b, const double2* Q, const double2* W, const int* order,
                              double2* U, cudaStream_t st) {
  note_launches(1); k_eig_rotate<<<dim3(128, g.G), 256, 0, st>>>(g.ns, b, Q, W, order, U);
  return cudaGetLastError();
}

// resid[g] = max_{r < keep_g} || (P U)[:, r] - lambda_r U[:, r] || / lambda_0
__global__ void k_eig_residual(int ns, int b, const int* __restrict__ keep, const double2* __restrict__ PU,
                               const double2* __restrict__ U, const double* __restrict__ ritz,
                               const int* __restrict__ order, double* __restrict__ resid) {
  __shared__ double red[32];
  const int grp = blockIdx.x;
  const size_t n = (size_t)ns * b;
  const double lam0 = ritz[(size_t)grp * b + order[(size_t)grp * b]];
  double worst = 0.0;
  for (int r = 0; r < keep[grp]; ++r) {
    const double lam = ritz[(size_t)grp * b + order[(size_t)grp * b + r]];
    double s = 0.0;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const double2 a = PU[(size_t)grp * n + (size_t)i * b + r];
      const double2 u = U[(size_t)grp * n + (size_t)i * b + r];
      const double dx = a.x - lam * u.x, dy = a.y - lam * u.y;
      s += dx * dx + dy * dy;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) worst = fmax(worst, sqrt(s) / fmax(fabs(lam0), 1e-300));
    __syncthreads();
  }
  if (threadIdx.x == 0) resid[grp] = worst;
}

cudaError_t launch_eig_residual(const Geo& g, int b, const double2* PU, const double2* U, const double* ritz,
                                const int* order, double* resid, cudaStream_t st) {
  note_launches(1); k_eig_residual<<<g.G, 256, 0, st>>>(g.ns, b, g.keep, PU, U, ritz, order, resid);
  return cudaGetLastError();
}

// A[aoff[g] + k ns + i] = sum_{n'} conj(U[(n',tau)][k]) T[n'][n], i = n w + tau
// (T = identity when null); AT is the same matrix stored [i][k].
// scale[g] = max |Re|, |Im| over A_g (per-group scale of the reduced-precision copies).
__global__ void k_form_A(Geo g, int b, const double2* __restrict__ U, const float2* __restrict__ T,
                         float2* __restrict__ A, float2* __restrict__ AT, float* __restrict__ scale) {
  __shared__ float red[32];
  const int grp = blockIdx.x;
  const int kg = g.keep[grp];
  const int base = g.aoff[grp];
  const double2* Ug = U + (size_t)grp * g.ns * b;
  float mx = 0.f;
  for (int o = threadIdx.x; o < kg * g.ns; o += blockDim.x) {
    const int k = o / g.ns, i = o - k * g.ns;
    const int n = i / g.w, tau = i - n * g.w;
    double re, im;
    if (T == nullptr) {
      const double2 u = Ug[(size_t)i * b + k];
      re = u.x;
      im = -u.y;
    } else {
      re = 0.0;
      im = 0.0;
      for (int m = 0; m < g.nc; ++m) {
        const double2 u = Ug[(size_t)(m * g.w + tau) * b + k];
        const float2 t = T[m * g.nc + n];
        // conj(u) * t
        re += u.x * t.x + u.y * t.y;
        im += u.x * t.y - u.y * t.x;
      }
    }
    const float2 v = make_float2((float)re, (float)im);
    A[base + (size_t)k * g.ns + i] = v;
    AT[base + (size_t)i * kg + k] = v;
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    scale[grp] = m;
  }
}

cudaError_t launch_form_A(const Geo& g, int b, const double2* U, const float2* T, float2* A, float2* AT,
                          float* scale, cudaStream_t st) {
  note_launches(1); k_form_A<<<g.G, 256, 0, st>>>(g, b, U, T, A, AT, scale);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ compress --
// S [lines][nc][ntx] -> Sc [lines][ntxc]; one block per (line, slab of kPB
// patches); the slab's samples of each coil are staged in shared memory.
constexpr int kPB = 32;
template <int MAXJ>
__global__ void __launch_bounds__(256) k_compress_fp32(Geo g, const float2* __restrict__ S,
                                                       const float2* __restrict__ AT, float2* __restrict__ Sc) {
  extern __shared__ float2 csm[];
  const int line = blockIdx.x;
  const int p0 = blockIdx.y * kPB;
  const int p1 = min(g.np, p0 + kPB);
  const int t0 = p0 * g.w, t1 = p1 * g.w;
  const int o0 = g.poff[p0];
  const int o1 = (p1 < g.np) ? g.poff[p1] : g.ntxc;
  float2 acc[MAXJ];
  int tb[MAXJ], ab[MAXJ], st[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    acc[j] = make_float2(0.f, 0.f);
    const int o = o0 + threadIdx.x + j * 256;
    tb[j] = o < o1 ? g.out_tbase[o] - t0 : 0;
    ab[j] = o < o1 ? g.out_abase[o] : 0;
    st[j] = o < o1 ? g.out_astride[o] : 0;
  }
  const float2* Sl = S + (size_t)line * g.nc * g.ntx;
  for (int n = 0; n < g.nc; ++n) {
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) csm[t - t0] = Sl[(size_t)n * g.ntx + t];
    __syncthreads();
    const int nw = n * g.w;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int o = o0 + threadIdx.x + j * 256;
      if (o < o1) {
        const float2* Ap = AT + ab[j] + (size_t)nw * st[j];
        for (int tau = 0; tau < g.w; ++tau) cfma(acc[j], __ldg(Ap + (size_t)tau * st[j]), csm[tb[j] + tau]);
      }
    }
    __syncthreads();
  }
  float2* out = Sc + (size_t)line * g.ntxc;
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    const int o = o0 + threadIdx.x + j * 256;
    if (o < o1) out[o] = acc[j];
  }
}

cudaError_t launch_compress_fp32(const Geo& g, const float2* S, int n_lines_in, const float2* AT, float2* Sc,
                                 cudaStream_t st) {
  const int nslab = (g.np + kPB - 1) / kPB;
  const size_t sm = sizeof(float2) * (size_t)kPB * g.w;
  const int need = (kPB * g.keep_max + 255) / 256;
  dim3 grid(n_lines_in, nslab);
#define KC(J)                                                                    \
  {                                                                              \
    cudaFuncSetAttribute(k_compress_fp32<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    note_launches(1); k_compress_fp32<J><<<grid, 256, sm, st>>>(g, S, AT, Sc);                     \
    return cudaGetLastError();                                                   \
  }
  if (need <= 1) KC(1)
  if (need <= 2) KC(2)
  if (need <= 4) KC(4)
  if (need <= 8) KC(8)
  if (need <= 16) KC(16)
#undef KC
  return cudaErrorInvalidValue;
}

}  // namespace gpjc
