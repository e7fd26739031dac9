// Two-pass batched FFT in shared memory for the transform lengths of the
// readout (N_x) and phase-encode (N_y, N_z) DFTs: n = N1 * N2 with N1 a power
// of two (16 or 8) and N2 <= 20 with prime factors 2, 3, 5, 7.
//
//   X[k1 + N1 k2] = sum_{i2} W_N2^{i2 k2} W_n^{i2 k1} sum_{i1} W_N1^{i1 k1} x[N2 i1 + i2]
//
// Pass 1: one thread per (transform, i2) loads the N1 elements x[N2 i1 + i2]
// into registers, computes their N1-point DFT, applies the twiddles W_n^{i2 k1}
// (table tw2[k1 N2 + i2], consecutive across threads) and stores the column to
// a scratch buffer with an XOR swizzle (row i2, column k1 ^ (i2 mod N1)), so
// that both the column-wise stores and the row-wise loads of pass 2 are free
// of bank conflicts.  Pass 2: one thread per (transform, k1) loads the N2
// values of its row, computes their N2-point DFT and writes X[k1 + N1 k2].
// The register DFTs are mixed-radix Cooley-Tukey with compile-time twiddles,
// so no index arithmetic is left at run time beyond divisions by constants.
// The result replaces the input in `a`; `b` holds batch * n scratch values.
#pragma once
#include <utility>

namespace gpjc {

// ---------------------------------------------------- compile-time trig --
// cos / sin of 2 pi p / q in double precision: quadrant reduction, then the
// Taylor series on [0, pi/2) (truncation below 1e-20).
namespace ct {
constexpr double kTwoPi = 6.28318530717958647692528676655900577;
__host__ __device__ constexpr double sin_poly(double x) {
  double x2 = x * x, t = x, s = x;
  for (int k = 1; k < 16; ++k) {
    t *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double cos_poly(double x) {
  double x2 = x * x, t = 1.0, s = 1.0;
  for (int k = 1; k < 16; ++k) {
    t *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double cos_turn(long p, long q) {
  const long m = ((p % q) + q) % q;
  const long quad = (4 * m) / q;
  const double th = (double)(4 * m - quad * q) / (4.0 * (double)q) * kTwoPi;
  const double c = cos_poly(th), s = sin_poly(th);
  return quad == 0 ? c : quad == 1 ? -s : quad == 2 ? -c : s;
}
__host__ __device__ constexpr double sin_turn(long p, long q) {
  const long m = ((p % q) + q) % q;
  const long quad = (4 * m) / q;
  const double th = (double)(4 * m - quad * q) / (4.0 * (double)q) * kTwoPi;
  const double c = cos_poly(th), s = sin_poly(th);
  return quad == 0 ? s : quad == 1 ? c : quad == 2 ? -s : -c;
}
}  // namespace ct

// compile-time loop: f(std::integral_constant<int, 0>) ... f(<N - 1>)
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// first factor of a composite register-DFT length
__host__ __device__ constexpr int dft_first_factor(int r) {
  return (r % 4 == 0 && r != 4 && r != 8) ? 4 : (r % 2 == 0) ? 2 : (r % 3 == 0) ? 3 : (r % 5 == 0) ? 5 : r;
}

// In-register R-point DFT, v[q] <- sum_r v[r] exp(SIGN 2 pi i r q / R).
template <int R, int SIGN>
__device__ __forceinline__ void dftr(float2* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<SIGN>(v);
  } else if constexpr (R == 3) {
    dft3<SIGN>(v);
  } else if constexpr (R == 4) {
    dft4<SIGN>(v);
  } else if constexpr (R == 5) {
    dft5<SIGN>(v);
  } else if constexpr (R == 7) {
    dft7<SIGN>(v);
  } else if constexpr (R == 8) {
    dft8<SIGN>(v);
  } else {
    constexpr int A = dft_first_factor(R), B = R / A;
    static_assert(A > 1 && B > 1 && A * B == R, "unsupported register DFT length");
    float2 t[R];
    // R = A B: DFT_A over the stride-B subsequences, twiddle, DFT_B
    static_for<B>([&](auto i2c) {
      constexpr int i2 = decltype(i2c)::value;
      float2 u[A];
      static_for<A>([&](auto i1c) { u[decltype(i1c)::value] = v[B * decltype(i1c)::value + i2]; });
      dftr<A, SIGN>(u);
      static_for<A>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        constexpr int m = (i2 * k1) % R;
        if constexpr (m == 0) {
          t[i2 * A + k1] = u[k1];
        } else {
          constexpr float c = (float)ct::cos_turn(m, R);
          constexpr float s = (float)(SIGN * ct::sin_turn(m, R));
          t[i2 * A + k1] = cmul(u[k1], make_float2(c, s));
        }
      });
    });
    static_for<A>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      float2 u[B];
      static_for<B>([&](auto i2c) { u[decltype(i2c)::value] = t[decltype(i2c)::value * A + k1]; });
      dftr<B, SIGN>(u);
      static_for<B>([&](auto k2c) { v[k1 + A * decltype(k2c)::value] = u[decltype(k2c)::value]; });
    });
  }
}

// Two-pass transform of `batch` sequences of length N1 N2 whose starts are
// `bs` elements apart in `a` (element i of the logical buffer at spad(i) when
// PAD).  tw2[k1 N2 + i2] = exp(-2 pi i i2 k1 / n).  Ends with __syncthreads().
template <int N1, int N2, int SIGN, bool PAD>
__device__ __forceinline__ void fft2p(float2* a, float2* b, int batch, int bs, const float2* __restrict__ tw2,
                                      int tid, int nthr) {
  constexpr int n = N1 * N2;
  static_assert((N1 & (N1 - 1)) == 0, "N1 must be a power of two");
  for (int task = tid; task < batch * N2; task += nthr) {
    const int f = task / N2, i2 = task - f * N2;
    const int base = f * bs + i2;
    float2 u[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) {
      const int li = base + N2 * i1;
      u[i1] = a[PAD ? spad(li) : li];
    }
    dftr<N1, SIGN>(u);
    float2* col = b + f * n + i2 * N1;
    const int sw = i2 & (N1 - 1);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 x = u[k1];
      if (k1 > 0) {
        float2 w = tw2[k1 * N2 + i2];
        if (SIGN > 0) w.y = -w.y;
        x = cmul(x, w);
      }
      col[k1 ^ sw] = x;
    }
  }
  __syncthreads();
  for (int task = tid; task < batch * N1; task += nthr) {
    const int f = task / N1, k1 = task - f * N1;
    float2 u[N2];
#pragma unroll
    for (int i2 = 0; i2 < N2; ++i2) u[i2] = b[f * n + i2 * N1 + (k1 ^ (i2 & (N1 - 1)))];
    dftr<N2, SIGN>(u);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int lo = f * bs + k1 + N1 * k2;
      a[PAD ? spad(lo) : lo] = u[k2];
    }
  }
  __syncthreads();
}

// Two-pass transform with caller-supplied input and output: ld(f, i) returns
// element i of transform f, st(f, k, v) receives element k (pre- and
// post-multiplications fuse into the two passes).  `b` holds batch * n
// scratch values; ends with __syncthreads().
template <int N1, int N2, int SIGN, typename LD, typename ST>
__device__ __forceinline__ void fft2p_cb(LD& ld, ST& st, float2* b, int batch, const float2* __restrict__ tw2,
                                         int tid, int nthr) {
  constexpr int n = N1 * N2;
  for (int task = tid; task < batch * N2; task += nthr) {
    const int f = task / N2, i2 = task - f * N2;
    float2 u[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) u[i1] = ld(f, N2 * i1 + i2);
    dftr<N1, SIGN>(u);
    float2* col = b + f * n + i2 * N1;
    const int sw = i2 & (N1 - 1);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 x = u[k1];
      if (k1 > 0) {
        float2 w = tw2[k1 * N2 + i2];
        if (SIGN > 0) w.y = -w.y;
        x = cmul(x, w);
      }
      col[k1 ^ sw] = x;
    }
  }
  __syncthreads();
  for (int task = tid; task < batch * N1; task += nthr) {
    const int f = task / N1, k1 = task - f * N1;
    float2 u[N2];
#pragma unroll
    for (int i2 = 0; i2 < N2; ++i2) u[i2] = b[f * n + i2 * N1 + (k1 ^ (i2 & (N1 - 1)))];
    dftr<N2, SIGN>(u);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) st(f, k1 + N1 * k2, u[k2]);
  }
  __syncthreads();
}

template <int SIGN, typename LD, typename ST>
__device__ __forceinline__ bool fft2p_cb_dispatch(int n1, int n2, LD& ld, ST& st, float2* b, int batch,
                                                  const float2* tw2, int tid, int nthr) {
  switch (fft2p_code(n1, n2)) {
    case fft2p_code(16, 8): fft2p_cb<16, 8, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 10): fft2p_cb<16, 10, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 12): fft2p_cb<16, 12, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 14): fft2p_cb<16, 14, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 15): fft2p_cb<16, 15, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 16): fft2p_cb<16, 16, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 18): fft2p_cb<16, 18, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(16, 20): fft2p_cb<16, 20, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(8, 5): fft2p_cb<8, 5, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    case fft2p_code(8, 7): fft2p_cb<8, 7, SIGN>(ld, st, b, batch, tw2, tid, nthr); return true;
    default: return false;
  }
}

// Runs the two-pass plan (n1, n2); false if the pair has no instantiation.
template <int SIGN, bool PAD>
__device__ __forceinline__ bool fft2p_dispatch(int n1, int n2, float2* a, float2* b, int batch, int bs,
                                               const float2* tw2, int tid, int nthr) {
  switch (fft2p_code(n1, n2)) {
    case fft2p_code(16, 8): fft2p<16, 8, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 10): fft2p<16, 10, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 12): fft2p<16, 12, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 14): fft2p<16, 14, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 15): fft2p<16, 15, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 16): fft2p<16, 16, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 18): fft2p<16, 18, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(16, 20): fft2p<16, 20, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(8, 5): fft2p<8, 5, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    case fft2p_code(8, 7): fft2p<8, 7, SIGN, PAD>(a, b, batch, bs, tw2, tid, nthr); return true;
    default: return false;
  }
}

}  // namespace gpjc
