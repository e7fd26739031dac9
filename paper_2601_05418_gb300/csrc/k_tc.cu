// Tensor-core (tcgen05) group compression and its adjoint, 16-bit operands
// (BF16 or FP16) with FP32 accumulation in tensor memory (Eq. 13-15).
//
// Complex products are embedded in real GEMMs with the contraction index
// interleaved as (sample i, re/im) -- the natural memory order of complex
// data -- and the output index interleaved as (k, re/im):
//   D[col][2k + c'] = sum_{i,c} X[col][2i + c] B[2i + c][2k + c'],
// B = [[Re A, Im A], [-Im A, Re A]] per (i, k).  For the compression
// (S' = A_g s, Eq. 13) a block owns 128 columns (lines x occurrences of
// group g); the patch samples of a chunk of coils are staged by one 4D TMA
// copy per chunk (periodic view [line][coil][occurrence][period]),
// converted to the no-swizzle K-major core-matrix layout, and one thread
// issues the MMAs (M = 128, N = 2 keep rounded to 16, K = 16 per
// instruction) into a TMEM accumulator that the four warps read back.
// B is pre-packed in global memory in the exact shared-memory image and
// copied with one bulk copy per chunk.  A per-group scale maps A_g to
// [-1, 1] before rounding and is re-applied in the epilogue.
//
// The adjoint (A_g^H applied to the compressed columns) is the same GEMM
// with the roles of k and i exchanged and N tiled by 256.
//
// BF16 (8 mantissa bits) runs split: every operand value v is carried as a
// head h = bf16(v) and a remainder l = bf16(v - h), and each K step issues
// three MMAs into the same accumulator (h_X h_B + l_X h_B + h_X l_B), so the
// products keep about 16 mantissa bits and the image stays within the
// FP32-path error of the oracle; FP16 (11 bits) runs one MMA per K step.
//
// Every wait on an mbarrier is bounded; on timeout the block records
// kDevTimeout in the status word, drains what it issued (again bounded),
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kTcThreads = 128;
// a wait gives up after about half a second of SM clock cycles
constexpr long long kWaitCycles = 1000000000ll;

// ------------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 > kWaitCycles) return false;
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
}
// The same wait taken by every thread of the block, with a block-uniform
// verdict (so that no thread leaves a loop whose barriers the others reach).
// The parity is flipped only on success: after a timeout it still names the
// operation in flight, which the block then drains before freeing TMEM.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t& parity) {
  const bool ok = __syncthreads_and(mbar_wait(bar, parity) ? 1 : 0) != 0;
  if (ok) parity ^= 1;
  return ok;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = (uint64_t)(smem_u32(p) & 0x3FFFF) >> 4;
  return a | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
         ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulate, A/B both FP16
// (fmt 0) or both BF16 (fmt 1), both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int n) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16-bit element conversions
template <int FMT>
__device__ __forceinline__ uint32_t pack2(float a, float b);
template <>
__device__ __forceinline__ uint32_t pack2<1>(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack2<0>(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <int FMT>
__device__ __forceinline__ float2 unpack2(uint32_t v);
template <>
__device__ __forceinline__ float2 unpack2<1>(uint32_t v) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
  return __bfloat1622float2(h);
}
template <>
__device__ __forceinline__ float2 unpack2<0>(uint32_t v) {
  __half2 h = *reinterpret_cast<__half2*>(&v);
  return __half22float2(h);
}

// element offset of (row, k) in a no-swizzle K-major core-matrix image with
// Kt columns (Kt multiple of 8)
__host__ __device__ __forceinline__ int core_off(int row, int k, int Kt) {
  return (row >> 3) * (Kt << 3) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// 16-bit images per operand: 2 (head + remainder) for BF16, 1 for FP16
__host__ __device__ constexpr int tc_images(int fmt) { return fmt == 1 ? 2 : 1; }
// elements of one group's expansion images (tiles of 256 rows, each tile
// its head image and, for BF16, its remainder image)
__host__ __device__ inline size_t tc_exp_group_elems(const TcGeom& t, int fmt) {
  return (size_t)((t.nexp + 255) / 256) * tc_images(fmt) * 256 * t.Kx;
}

// ------------------------------------------------------------------ packing --
// Compression B per (group, coil chunk): rows 2k + c' (N), columns
// 2 (n_local w + tau) + c (K), core-matrix image, values of A_g / scale_g.
template <int FMT>
__global__ void k_tc_pack_comp(TcGeom t, const float2* __restrict__ A, const float* __restrict__ scale,
                               uint16_t* __restrict__ B) {
  const int g = blockIdx.y, chunk = blockIdx.z;
  const size_t per = (size_t)t.npad * t.Kc;
  // head image, then (BF16) the remainder image of the same (group, chunk)
  uint16_t* Bg = B + ((size_t)g * t.nchunks + chunk) * per * tc_images(FMT);
  const float inv = scale[g] > 0.f ? 1.0f / scale[g] : 0.f;
  const int keep = t.keep[g];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < t.npad * t.Kc; idx += gridDim.x * blockDim.x) {
    const int nr = idx / t.Kc, kk = idx - nr * t.Kc;
    const int kout = nr >> 1, cout = nr & 1;
    const int nl = kk / (2 * t.w), rem = kk - nl * 2 * t.w;
    const int tau = rem >> 1, cin = rem & 1;
    const int n = chunk * t.ncc + nl;
    float v = 0.f;
    if (kout < keep && n < t.nc && nl < t.ncc) {
      const float2 a = A[t.aoff[g] + (size_t)kout * t.ns + n * t.w + tau];
      const float re = a.x * inv, im = a.y * inv;
      v = (cin == 0) ? (cout == 0 ? re : im) : (cout == 0 ? -im : re);
    }
    const uint32_t p = pack2<FMT>(v, 0.f);
    Bg[core_off(nr, kk, t.Kc)] = (uint16_t)(p & 0xFFFF);
    if (tc_images(FMT) == 2) Bg[per + core_off(nr, kk, t.Kc)] = (uint16_t)(pack2<FMT>(v - unpack2<FMT>(p).x, 0.f) & 0xFFFF);
  }
}

// Expansion B per (group, N tile of 256): rows 2 i + c (N, i = n w + tau),
// columns 2 k + c' (K, padded to Kx), values of conj(A_g)^T / scale_g:
//   U_i = sum_k conj(A_ki) h_k  ->  [Re U; Im U] from [Re h; Im h].
template <int FMT>
__global__ void k_tc_pack_exp(TcGeom t, const float2* __restrict__ A, const float* __restrict__ scale,
                              uint16_t* __restrict__ B) {
  const int g = blockIdx.y;
  const int nimg = tc_images(FMT);
  uint16_t* Bg = B + (size_t)g * tc_exp_group_elems(t, FMT);
  const float inv = scale[g] > 0.f ? 1.0f / scale[g] : 0.f;
  const int keep = t.keep[g];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < t.nexp * t.Kx; idx += gridDim.x * blockDim.x) {
    const int nr = idx / t.Kx, kk = idx - nr * t.Kx;
    const int i = nr >> 1, c = nr & 1;      // output sample and re/im
    const int k = kk >> 1, cp = kk & 1;      // input kept component and re/im
    float v = 0.f;
    if (i < t.ns && k < keep) {
      const float2 a = A[t.aoff[g] + (size_t)k * t.ns + i];
      const float re = a.x * inv, im = a.y * inv;
      // Re U = Re A Re h + Im A Im h ; Im U = Re A Im h - Im A Re h
      v = (c == 0) ? (cp == 0 ? re : im) : (cp == 0 ? -im : re);
    }
    // N tiles of 256 rows are stored one after another, each its own image
    // (BF16: the tile's head image, then its remainder image)
    const int tile = nr >> 8, rr = nr & 255;
    uint16_t* Bt = Bg + (size_t)tile * nimg * 256 * t.Kx;
    const uint32_t p = pack2<FMT>(v, 0.f);
    Bt[core_off(rr, kk, t.Kx)] = (uint16_t)(p & 0xFFFF);
    if (nimg == 2) Bt[256 * t.Kx + core_off(rr, kk, t.Kx)] = (uint16_t)(pack2<FMT>(v - unpack2<FMT>(p).x, 0.f) & 0xFFFF);
  }
}

// ------------------------------------------------------------------ compression GEMM --
// Source element: float (SRC_BYTES = 4, converted) or the 16-bit operand
// type itself (SRC_BYTES = 2).  Output: out[line][off_p + k] complex64.
template <int FMT, int SRC_BYTES>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_compress(const __grid_constant__ CUtensorMap tmap, TcGeom t,
                                                              const uint16_t* __restrict__ Bpk,
                                                              float2* __restrict__ out, int line0,
                                                              int n_lines, int* status) {
  // BF16 splits the FP32 source into head + remainder (16-bit sources are FP16 only)
  static_assert(FMT == 0 || SRC_BYTES == 4, "the BF16 compression takes FP32 sources");
  constexpr int NI = tc_images(FMT);
  extern __shared__ __align__(1024) unsigned char tsm[];
  const int g = blockIdx.y;
  const int l0 = line0 + blockIdx.x * t.lt;
  unsigned char* stg = tsm;                                   // staging [lt][ncc][n_occ][box0]
  uint16_t* At = (uint16_t*)(tsm + t.stg_bytes);              // 128 x Kc core image (head)
  uint16_t* Al = At + (NI - 1) * 128 * t.Kc;                  // 128 x Kc remainder (BF16)
  uint16_t* Bt0 = Al + 128 * t.Kc;                            // npad x Kc core image(s) of A_g, two buffers
  const size_t bsz = (size_t)NI * t.npad * t.Kc;
  uint64_t* bars = (uint64_t*)(Bt0 + 2 * bsz);                // [0] load, [1] mma
  uint32_t* tmem_slot = (uint32_t*)(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, t.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_f16(FMT, t.npad);
  const int x0 = ((2 * g * t.w) / t.xalign) * t.xalign;
  const int shift = 2 * g * t.w - x0;
  const uint32_t bbytes = (uint32_t)(NI * t.npad * t.Kc * 2);
  uint32_t ph_ld = 0, ph_mma = 0;
  bool ok = true;
  const int m = tid;  // A row = output column (line l, occurrence q); rows >= lt n_occ are padding
  const bool mrow = m < t.lt * t.n_occ;
  const int l = mrow ? m / t.n_occ : 0, q = mrow ? m - (m / t.n_occ) * t.n_occ : 0;
  // Chunk c + 1's staging and A_g image are loaded while chunk c's MMAs run:
  // its staging load is issued once the block has converted chunk c's
  // staging (block barrier), into the same buffer; its A_g image goes to the
  // other of two buffers, which chunk c - 1's MMAs (waited for) no longer
  // read.  The images of chunk c + 1 are written only after chunk c's MMAs
  // have completed.
  bool ld_pending = false, mma_pending = false;
  if (tid == 0) {
    mbar_expect_tx(&bars[0], (uint32_t)t.stg_tx + bbytes);
    tma_load_4d(stg, &tmap, x0, 0, 0, l0, &bars[0]);
    bulk_g2s(Bt0, Bpk + (size_t)g * t.nchunks * bsz, bbytes, &bars[0]);
  }
  ld_pending = true;
  for (int c = 0; c < t.nchunks && ok; ++c) {
    uint16_t* Bt = Bt0 + (size_t)(c & 1) * bsz;
    if (!(ok = block_wait(&bars[0], ph_ld))) break;
    ld_pending = false;
    // staging -> 16-bit core image (row m holds its column's samples of the chunk)
    for (int nl = 0; nl < t.ncc && mrow; ++nl) {
      const size_t base = ((size_t)(l * t.ncc + nl) * t.n_occ + q) * t.box0 + shift;
      for (int tau = 0; tau < t.w; ++tau) {
        uint32_t pk, pl = 0u;
        if (SRC_BYTES == 4) {
          const float* s = (const float*)stg + base + 2 * tau;
          pk = pack2<FMT>(s[0], s[1]);
          if (NI == 2) {
            const float2 h = unpack2<FMT>(pk);
            pl = pack2<FMT>(s[0] - h.x, s[1] - h.y);
          }
        } else {
          const uint16_t* s = (const uint16_t*)stg + base + 2 * tau;
          pk = (uint32_t)s[0] | ((uint32_t)s[1] << 16);
        }
        const int k = 2 * (nl * t.w + tau);
        *(uint32_t*)(At + core_off(m, k, t.Kc)) = pk;
        if (NI == 2) *(uint32_t*)(Al + core_off(m, k, t.Kc)) = pl;
      }
    }
    for (int k = mrow ? 2 * t.ncc * t.w : 0; k < t.Kc; k += 2) {
      *(uint32_t*)(At + core_off(m, k, t.Kc)) = 0u;
      if (NI == 2) *(uint32_t*)(Al + core_off(m, k, t.Kc)) = 0u;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (c + 1 < t.nchunks) {
      if (tid == 0) {
        mbar_expect_tx(&bars[0], (uint32_t)t.stg_tx + bbytes);
        tma_load_4d(stg, &tmap, x0, 0, (c + 1) * t.ncc, l0, &bars[0]);
        bulk_g2s(Bt0 + (size_t)((c + 1) & 1) * bsz, Bpk + ((size_t)g * t.nchunks + c + 1) * bsz, bbytes,
                 &bars[0]);
      }
      ld_pending = true;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sbo = (uint32_t)(t.Kc / 8) * 128;
      for (int ks = 0; ks < t.Kc / 16; ++ks) {
        const uint64_t ad = umma_desc(At + ks * 16 * 8, 128, sbo);
        const uint64_t bd = umma_desc(Bt + ks * 16 * 8, 128, sbo);
        mma_f16(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
        if (NI == 2) {
          // remainder x head and head x remainder into the same accumulator
          mma_f16(tmem, umma_desc(Al + ks * 16 * 8, 128, sbo), bd, idesc, 1u);
          mma_f16(tmem, ad, umma_desc(Bt + (size_t)t.npad * t.Kc + ks * 16 * 8, 128, sbo), idesc, 1u);
        }
      }
      mma_commit(&bars[1]);
    }
    mma_pending = true;
    if (!(ok = block_wait(&bars[1], ph_mma))) break;
    mma_pending = false;
  }
  if (!ok) {
    if (tid == 0) atomicExch(status, (int)kDevTimeout);
    // drain the operations still in flight before releasing the memory
    if (ld_pending) mbar_wait(&bars[0], ph_ld);
    if (mma_pending) mbar_wait(&bars[1], ph_mma);
  } else {
    tc_fence_after();
    // epilogue: lane m of TMEM holds column m; 8 fp32 columns = 4 complex values per load
    const int line = l0 + l;
    const int p = (g * t.w + q * t.P) / t.w;
    const bool valid = mrow && line < n_lines;
    const float s = t.scale[g];
    const int keep = t.keep[g];
    float2* o = out + (size_t)line * t.ntxc + (valid ? t.poff[p] : 0);
    for (int col = 0; col < t.npad; col += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = col / 2 + j;
          if (k < keep) o[k] = make_float2(v[2 * j] * s, v[2 * j + 1] * s);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, t.tmem_cols);
}

// ------------------------------------------------------------------ expansion GEMM --
// V[row][n][p w + tau] = sum_k conj(A_g[k][n w + tau]) H[row][off_p + k],
// FP32 output.  A block owns 128 columns (rows x occurrences of g).  The
// FP32 input column is split into a 16-bit head and a 16-bit remainder
// (two MMAs into the same accumulator), so only A_g is rounded to 16 bits:
// rounding the compressed hybrid data itself would break the adjoint
// pairing that CG relies on far more than rounding the matrix does.
template <int FMT>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_expand(TcGeom t, const float2* __restrict__ H,
                                                            const uint16_t* __restrict__ Bpk,
                                                            float2* __restrict__ V, int n_rows, int* status) {
  constexpr int NI = tc_images(FMT);
  extern __shared__ __align__(1024) unsigned char tsm[];
  const int g = blockIdx.y;
  const int r0 = blockIdx.x * t.lt;
  uint16_t* Ah = (uint16_t*)tsm;                        // 128 x Kx head
  uint16_t* Al = Ah + 128 * t.Kx;                       // 128 x Kx remainder
  uint16_t* Bt = Al + 128 * t.Kx;                       // 256 x Kx head (+ 256 x Kx remainder, BF16)
  uint64_t* bars = (uint64_t*)(Bt + NI * 256 * t.Kx);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, 256);
  const int m = tid;  // rows >= lt n_occ of the tile are padding
  const bool mrow = m < t.lt * t.n_occ;
  const int l = mrow ? m / t.n_occ : 0, q = mrow ? m - (m / t.n_occ) * t.n_occ : 0;
  const int row = r0 + l;
  const int p = (g * t.w + q * t.P) / t.w;
  const bool valid = mrow && row < n_rows;
  const int keep = t.keep[g];
  const float2* h = H + (size_t)(valid ? row : 0) * t.ntxc + t.poff[p];
  for (int k = 0; k < t.Kx / 2; ++k) {
    const float2 v = (valid && k < keep) ? h[k] : make_float2(0.f, 0.f);
    const uint32_t hi = pack2<FMT>(v.x, v.y);
    const float2 hv = unpack2<FMT>(hi);
    *(uint32_t*)(Ah + core_off(m, 2 * k, t.Kx)) = hi;
    *(uint32_t*)(Al + core_off(m, 2 * k, t.Kx)) = pack2<FMT>(v.x - hv.x, v.y - hv.y);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const float s = t.scale[g];
  uint32_t ph_ld = 0, ph_mma = 0;
  bool ok = true;
  uint64_t* stuck = nullptr;
  const int ntiles = (t.nexp + 255) / 256;
  for (int nt = 0; nt < ntiles && ok; ++nt) {
    const int nrows = min(256, t.nexp - nt * 256);  // multiple of 16
    const uint32_t bbytes = (uint32_t)(nrows * t.Kx * 2);
    if (tid == 0) {
      const uint16_t* src = Bpk + (size_t)g * tc_exp_group_elems(t, FMT) + (size_t)nt * NI * 256 * t.Kx;
      mbar_expect_tx(&bars[0], NI * bbytes);
      bulk_g2s(Bt, src, bbytes, &bars[0]);
      if (NI == 2) bulk_g2s(Bt + 256 * t.Kx, src + 256 * t.Kx, bbytes, &bars[0]);
    }
    if (!(ok = block_wait(&bars[0], ph_ld))) {
      stuck = &bars[0];
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sbo = (uint32_t)(t.Kx / 8) * 128;
      const uint32_t idesc = idesc_f16(FMT, nrows);
      for (int ks = 0; ks < t.Kx / 16; ++ks) {
        const uint64_t bd = umma_desc(Bt + ks * 16 * 8, 128, sbo);
        mma_f16(tmem, umma_desc(Ah + ks * 16 * 8, 128, sbo), bd, idesc, ks > 0 ? 1u : 0u);
        mma_f16(tmem, umma_desc(Al + ks * 16 * 8, 128, sbo), bd, idesc, 1u);
        if (NI == 2)  // head of H x remainder of A_g
          mma_f16(tmem, umma_desc(Ah + ks * 16 * 8, 128, sbo),
                  umma_desc(Bt + 256 * t.Kx + ks * 16 * 8, 128, sbo), idesc, 1u);
      }
      mma_commit(&bars[1]);
    }
    if (!(ok = block_wait(&bars[1], ph_mma))) {
      stuck = &bars[1];
      break;
    }
    tc_fence_after();
    for (int col = 0; col < nrows; col += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
      const int i0 = (nt * 256 + col) / 2;  // patch vector index n w + tau of v[0], a multiple of 4
      if (valid && (t.w & 3) == 0) {
        // the four samples share the coil n and start on a 32-byte boundary
        if (i0 < t.ns) {
          const int n = i0 / t.w, tau = i0 - n * t.w;
          float4* dst = reinterpret_cast<float4*>(V + ((size_t)row * t.nc + n) * t.ntx + p * t.w + tau);
          dst[0] = make_float4(v[0] * s, v[1] * s, v[2] * s, v[3] * s);
          dst[1] = make_float4(v[4] * s, v[5] * s, v[6] * s, v[7] * s);
        }
      } else if (valid) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = i0 + j;
          if (i < t.ns) {
            const int n = i / t.w, tau = i - n * t.w;
            V[((size_t)row * t.nc + n) * t.ntx + p * t.w + tau] = make_float2(v[2 * j] * s, v[2 * j + 1] * s);
          }
        }
      }
    }
    // all lanes must finish reading TMEM before the next tile's MMAs overwrite it
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (!ok) {
    if (tid == 0) atomicExch(status, (int)kDevTimeout);
    mbar_wait(stuck, stuck == &bars[0] ? ph_ld : ph_mma);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// ------------------------------------------------------------------ host side --
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 4D periodic view of [lines][nc][ntx] complex data with elements of
// `ebytes` (4 = float, 2 = 16-bit): dims (2P, n_occ, nc, lines).
bool make_tc_tmap(const TcGeom& t, const void* base, int lines, int ebytes, CUtensorMap* map) {
  auto enc = get_encode();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)(2 * t.P), (cuuint64_t)t.n_occ, (cuuint64_t)t.nc, (cuuint64_t)lines};
  const cuuint64_t strides[3] = {(cuuint64_t)(2 * t.P) * ebytes, (cuuint64_t)(2 * t.ntx) * ebytes,
                                 (cuuint64_t)t.nc * 2 * t.ntx * ebytes};
  const cuuint32_t box[4] = {(cuuint32_t)t.box0, (cuuint32_t)t.n_occ, (cuuint32_t)t.ncc, (cuuint32_t)t.lt};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(map, ebytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 4,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t tc_compress_smem(const TcGeom& t, int fmt) {
  const int ni = tc_images(fmt);
  // staging, the chunk's 16-bit images, two buffers of A_g images, barriers
  return (size_t)t.stg_bytes + (size_t)ni * 128 * t.Kc * 2 + (size_t)2 * ni * t.npad * t.Kc * 2 + 64;
}
size_t tc_expand_smem(const TcGeom& t, int fmt) {
  return (size_t)2 * 128 * t.Kx * 2 + (size_t)tc_images(fmt) * 256 * t.Kx * 2 + 64;
}
size_t tc_pack_comp_elems(const TcGeom& t, int fmt) {
  return (size_t)t.G * t.nchunks * t.npad * t.Kc * tc_images(fmt);
}
size_t tc_pack_exp_elems(const TcGeom& t, int fmt) { return (size_t)t.G * tc_exp_group_elems(t, fmt); }

cudaError_t launch_tc_pack(const TcGeom& t, int fmt, const float2* A, const float* scale, uint16_t* Bc,
                           uint16_t* Bx, cudaStream_t st) {
  dim3 gc(8, t.G, t.nchunks), gx(8, t.G);
  if (fmt == 1) {
    note_launches(1); k_tc_pack_comp<1><<<gc, 256, 0, st>>>(t, A, scale, Bc);
    note_launches(1); k_tc_pack_exp<1><<<gx, 256, 0, st>>>(t, A, scale, Bx);
  } else {
    note_launches(1); k_tc_pack_comp<0><<<gc, 256, 0, st>>>(t, A, scale, Bc);
    note_launches(1); k_tc_pack_exp<0><<<gx, 256, 0, st>>>(t, A, scale, Bx);
  }
  return cudaGetLastError();
}

template <int FMT, int SB>
static cudaError_t launch_comp_t(const CUtensorMap& map, const TcGeom& t, const uint16_t* Bc, float2* out,
                                 int line0, int lines, int* status, cudaStream_t st) {
  const size_t sm = tc_compress_smem(t, FMT);
  static size_t attr = 0;
  if (sm > attr) {
    cudaFuncSetAttribute(k_tc_compress<FMT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  dim3 grid((lines - line0 + t.lt - 1) / t.lt, t.G);
  note_launches(1); k_tc_compress<FMT, SB><<<grid, kTcThreads, sm, st>>>(map, t, Bc, out, line0, lines, status);
  return cudaGetLastError();
}

cudaError_t launch_tc_compress(const CUtensorMap& map, const TcGeom& t, int fmt, int src_bytes, const uint16_t* Bc,
                               float2* out, int line0, int lines, int* status, cudaStream_t st) {
  if (line0 < 0 || line0 >= lines || line0 % t.lt) return cudaErrorInvalidValue;
  if (fmt == 1 && src_bytes == 4) return launch_comp_t<1, 4>(map, t, Bc, out, line0, lines, status, st);
  if (fmt == 0 && src_bytes == 4) return launch_comp_t<0, 4>(map, t, Bc, out, line0, lines, status, st);
  if (fmt == 0 && src_bytes == 2) return launch_comp_t<0, 2>(map, t, Bc, out, line0, lines, status, st);
  return cudaErrorInvalidValue;
}

template <int FMT>
static cudaError_t launch_exp_t(const TcGeom& t, const float2* H, const uint16_t* Bx, float2* V, int rows,
                                int* status, cudaStream_t st) {
  const size_t sm = tc_expand_smem(t, FMT);
  static size_t attr = 0;
  if (sm > attr) {
    cudaFuncSetAttribute(k_tc_expand<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  dim3 grid((rows + t.lt - 1) / t.lt, t.G);
  note_launches(1); k_tc_expand<FMT><<<grid, kTcThreads, sm, st>>>(t, H, Bx, V, rows, status);
  return cudaGetLastError();
}

cudaError_t launch_tc_expand(const TcGeom& t, int fmt, const float2* H, const uint16_t* Bx, float2* V, int rows,
                             int* status, cudaStream_t st) {
  return fmt == 1 ? launch_exp_t<1>(t, H, Bx, V, rows, status, st) : launch_exp_t<0>(t, H, Bx, V, rows, status, st);
}

}  // namespace gpjc

// ====================================================================== Gram --
// P_g = sum_r v_r v_r^H on the tensor cores (Eq. 9-11).  Values are scaled by
// 2^12 and split into an FP16 head and remainder; three MMAs per K step (head
// x head, head x rest, rest x head) keep the products at about FP32 accuracy.
namespace gpjc {

constexpr float kTgScale = 4096.0f;  // 2^12 before the split; products carry 2^24

__device__ __forceinline__ void split_f16(float a, float b, uint32_t* hi, uint32_t* lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  *hi = *reinterpret_cast<const uint32_t*>(&h);
  *lo = *reinterpret_cast<const uint32_t*>(&l);
}

// ---------------------------------------------------------------- Gram (C x Psi) --
// The patch vector of pixel r is v_r = c_hat(r) (x) psi_g(r) (coil-major), so
//   P_g[(n, tau), (n', tau')] = sum_r C_{n n'}(r) Psi_{g tau tau'}(r),
//   C_{n n'} = c_hat_n conj(c_hat_n'),  Psi_{g tau tau'} = psi_{g tau} conj(psi_{g tau'}).
// One GEMM over the ROI pixels gives every group at once: M = coil pairs
// n <= n' (shared by all groups), N = (g, tau, tau') (shared by all coil
// pairs), so each operand value is generated once per pixel per tile instead
// of once per (row, column) tile of every P_g.  Real embedding as above
// (K = (pixel, re/im); B rows 2e = [Re Psi, -Im Psi], 2e+1 = [Im Psi, Re Psi]),
// FP16 head/remainder split (three MMAs per K step), 128 x 256 tiles with a
// 256-column TMEM accumulator, operand images double-buffered so that the
// eight warps build chunk c+1 while the MMAs of chunk c run.  FP32 runs of at
// most 256 pixels in the tensor memory are summed in registers, and a block
// adds its sums to P_g with FP64 atomics when its tile changes (persistent
// blocks over a tile-major split of the (tile, chunk) units).  Entries with
// n > n' are filled by the Hermitian completion.
constexpr int kTg2Threads = 512;          // 16 warps: 4 per TMEM lane quarter
constexpr int kTg2Cols = 256 * 128 / kTg2Threads;  // accumulator columns per thread (64)
constexpr int kTg2KC = 32;          // pixels per chunk (K = 64)
constexpr int kTg2Px = kTg2KC * 128 / kTg2Threads;  // pixels per thread per chunk (8)
constexpr int kTg2Run = 8;          // chunks per FP32 run in the tensor memory (256 pixels)
constexpr int kTg2PS = kTg2KC + 1;  // row stride of the phase table (odd: no bank conflicts)
constexpr int kTg2ImgA = 128 * 64;  // uint16 per A image
constexpr int kTg2ImgB = 256 * 64;  // uint16 per B image

__host__ __device__ inline int tg2_groups_per_tile(int w) {
  const int w2 = w * w;
  return (128 + w2 - 1) / w2 + 1;
}

// Tile-dependent operand rows of one thread.
struct Tg2Rows {
  int m, na, nb, e, gl, tau, taup, g_lo, ng;
  bool mval, eval;
};
__device__ __forceinline__ Tg2Rows tg2_rows(const Geo& g, const int2* __restrict__ cpairs, int npairs, int mt,
                                            int ntile, int row, int gpt) {
  Tg2Rows r;
  const int w = g.w, w2 = w * w, ne = g.G * w2;
  r.m = mt * 128 + row;
  r.mval = r.m < npairs;
  r.na = r.nb = 0;
  if (r.mval) {
    const int2 pr = cpairs[r.m];
    r.na = pr.x;
    r.nb = pr.y;
  }
  r.e = ntile * 128 + row;
  r.eval = r.e < ne;
  r.g_lo = (ntile * 128) / w2;
  const int ge = r.eval ? r.e / w2 : r.g_lo;
  const int rem = r.eval ? r.e - ge * w2 : 0;
  r.tau = rem / w;
  r.taup = rem - r.tau * w;
  r.gl = ge - r.g_lo;
  r.ng = min(gpt, g.G - r.g_lo);
  return r;
}

// Adds a tile's sums (this thread's TMEM lane row, kTg2Cols columns of the
// cross-run accumulator at tacc) to P_g.
__device__ __forceinline__ void tg2_flush(const Geo& g, const int2* __restrict__ cpairs, int npairs, int mt,
                                          int ntile, uint32_t tacc, double2* __restrict__ P) {
  const int warp = threadIdx.x >> 5;
  const int w = g.w, w2 = w * w, ne = g.G * w2;
  const double sc = 1.0 / ((double)kTgScale * (double)kTgScale);
  const int mrow = mt * 128 + (warp & 3) * 32 + (threadIdx.x & 31);
  const int colh = (warp >> 2) * kTg2Cols;
  const bool ok = mrow < npairs;
  const int2 pr = ok ? cpairs[mrow] : make_int2(0, 0);
  for (int col = 0; col < kTg2Cols; col += 8) {
    float v[8];
    tmem_ld8(tacc + (uint32_t)col, v);  // all lanes take part in the collective load
    if (!ok) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ee = ntile * 128 + (colh + col) / 2 + j;
      if (ee < ne) {
        const int gg = ee / w2, rr2 = ee - gg * w2;
        const int t1 = rr2 / w, t2 = rr2 - t1 * w;
        double2* d = P + ((size_t)gg * g.ns + (size_t)(pr.x * w + t1)) * g.ns + (pr.y * w + t2);
        atomicAdd(&d->x, (double)v[2 * j] * sc);
        atomicAdd(&d->y, (double)v[2 * j + 1] * sc);
      }
    }
  }
}

// Adds the finished FP32 run (TMEM columns at trun) to the cross-run
// accumulator (columns at tacc), or copies it there for a tile's first run.
__device__ __forceinline__ void tg2_fold(uint32_t trun, uint32_t tacc, bool first) {
  for (int col = 0; col < kTg2Cols; col += 8) {
    float v[8], a[8];
    tmem_ld8(trun + (uint32_t)col, v);
    if (!first) {
      tmem_ld8(tacc + (uint32_t)col, a);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] += a[q];
    }
    tmem_st8(tacc + (uint32_t)col, v);
  }
  tmem_wait_st();
}

// Persistent: the (tile, 32-pixel chunk) units, tile-major, are split into
// gridDim.x contiguous ranges (one per block), so each block sums long runs
// of one tile and adds to P_g only when its tile changes.
__global__ void __launch_bounds__(kTg2Threads, 1) k_tc_gram2(Geo g, const float2* __restrict__ chat,
                                                            const int* __restrict__ pix,
                                                            const int* __restrict__ dK, int Kpad,
                                                            const int* __restrict__ pref,
                                                            const int2* __restrict__ cpairs, int npairs,
                                                            int n_tiles, int n_ntiles, double2* __restrict__ P,
                                                            int* status) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  uint16_t* img = (uint16_t*)tsm;  // [buf][Ah, Al, Bh, Bl]
  const int gpt = tg2_groups_per_tile(g.w);
  float2* psi = (float2*)(img + 2 * (2 * kTg2ImgA + 2 * kTg2ImgB));  // [gl][tau][px], rows kTg2PS apart
  int4* pxy = (int4*)(((uintptr_t)(psi + gpt * g.w * kTg2PS) + 15) & ~(uintptr_t)15);  // chunk pixels (x, y, z, valid)
  uint64_t* bars = (uint64_t*)(pxy + kTg2KC);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2);
  const int w = g.w;
  const int K = *dK;
  const int nck = (K + kTg2KC - 1) / kTg2KC;
  const long long U = (long long)n_tiles * nck;
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  if (u0 >= u1) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_f16(0, 256);
  const uint32_t sbo = (64 / 8) * 128;
  const float inv_ny = 1.0f / (float)g.ny, inv_nz = 1.0f / (float)g.nz;
  const int row = tid & 127, quarter = tid >> 7;
  // this thread's share of the MMA accumulator (columns 0-255: one FP32 run
  // of at most kTg2Run chunks = 256 pixels) and of the cross-run FP32 sum
  // (columns 256-511): TMEM lane row, kTg2Cols columns
  const uint32_t tm_row = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * kTg2Cols);
  const uint32_t tm_acc = tm_row + 256u;
  bool acc_first = true;
  uint32_t par[2] = {0u, 0u};
  bool pend[2] = {false, false};
  bool ok = true;
  int c = 0, run = 0;
  int cur = -1;  // tile of the chunks in flight / in the registers
  Tg2Rows R;
  for (long long u = u0; u < u1; ++u, ++c) {
    const int tile = (int)(u / nck);
    const int k0 = (int)(u - (long long)tile * nck) * kTg2KC;
    const int buf = c & 1;
    uint16_t* Ah = img + buf * (2 * kTg2ImgA + 2 * kTg2ImgB);
    uint16_t* Al = Ah + kTg2ImgA;
    uint16_t* Bh = Al + kTg2ImgA;
    uint16_t* Bl = Bh + kTg2ImgB;
    if (pend[buf]) {  // the MMAs of chunk c - 2 read this buffer
      if (!(ok = block_wait(&bars[buf], par[buf]))) break;
      pend[buf] = false;
    }
    const int mt = tile / n_ntiles, ntile = tile - mt * n_ntiles;
    if (tile != cur) R = tg2_rows(g, cpairs, npairs, mt, ntile, row, gpt);
    // the chunk's pixel coordinates, then the phases psi_{g tau}(r) of the
    // tile's groups
    if (tid < kTg2KC) {
      const int k = k0 + tid;
      int4 q = make_int4(0, 0, 0, 0);
      if (k < K) {
        const int p = pix[k];
        const int rw = p / g.nx;
        q = make_int4(p - rw * g.nx - g.nx / 2, rw % g.ny - g.ny / 2, rw / g.ny - g.nz / 2, 1);
      }
      pxy[tid] = q;
    }
    __syncthreads();
    for (int idx = tid; idx < R.ng * w * kTg2KC; idx += kTg2Threads) {
      const int gt = idx / kTg2KC, r = idx - gt * kTg2KC;
      const int gg = R.g_lo + gt / w, tt = gt - (gt / w) * w;
      const int4 q = pxy[r];
      float2 ph = make_float2(0.f, 0.f);
      if (q.w) {
        const int t = pref[gg] * w + tt;
        int prod = ((t - g.ntx / 2) * q.x) % g.ntx;
        if (prod < 0) prod += g.ntx;
        const float wave = g.ay[t] * (float)q.y * inv_ny + (g.nz > 1 ? g.az[t] * (float)q.z * inv_nz : 0.0f);
        ph = expipi(-(2.0f * (float)prod / (float)g.ntx + 2.0f * wave));
      }
      psi[gt * kTg2PS + r] = ph;
    }
    __syncthreads();
    const float2* pa = psi + (R.gl * w + R.tau) * kTg2PS;
    const float2* pb = psi + (R.gl * w + R.taup) * kTg2PS;
    const float2* ca = chat + (size_t)R.na * Kpad + k0;
    const float2* cb = chat + (size_t)R.nb * Kpad + k0;
    // four pixels (8 K values = one 16-byte core-matrix row) per store; the
    // part-1 pair (Im Psi, Re Psi) is the part-0 pair (Re Psi, -Im Psi) with
    // its two halves swapped and the new first (low) half negated (FP16
    // rounding is symmetric, so head and remainder transform alike)
#pragma unroll 1
    for (int q4 = 0; q4 < kTg2Px / 4; ++q4) {
      const int r0 = quarter * kTg2Px + 4 * q4;
      uint32_t ah[4], al[4], b0h[4], b0l[4], b1h[4], b1l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = r0 + j;
        float2 cv = make_float2(0.f, 0.f), pv = make_float2(0.f, 0.f);
        if (R.mval) cv = cscale(cmulc(cb[r], ca[r]), kTgScale);
        if (R.eval) pv = cscale(cmulc(pb[r], pa[r]), kTgScale);
        split_f16(cv.x, cv.y, &ah[j], &al[j]);
        split_f16(pv.x, -pv.y, &b0h[j], &b0l[j]);
        b1h[j] = __byte_perm(b0h[j], 0, 0x1032) ^ 0x00008000u;
        b1l[j] = __byte_perm(b0l[j], 0, 0x1032) ^ 0x00008000u;
      }
      const int kk = 2 * r0;
      *(uint4*)(Ah + core_off(row, kk, 64)) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
      *(uint4*)(Al + core_off(row, kk, 64)) = make_uint4(al[0], al[1], al[2], al[3]);
      *(uint4*)(Bh + core_off(2 * row, kk, 64)) = make_uint4(b0h[0], b0h[1], b0h[2], b0h[3]);
      *(uint4*)(Bl + core_off(2 * row, kk, 64)) = make_uint4(b0l[0], b0l[1], b0l[2], b0l[3]);
      *(uint4*)(Bh + core_off(2 * row + 1, kk, 64)) = make_uint4(b1h[0], b1h[1], b1h[2], b1h[3]);
      *(uint4*)(Bl + core_off(2 * row + 1, kk, 64)) = make_uint4(b1l[0], b1l[1], b1l[2], b1l[3]);
    }
    // a run closes at kTg2Run chunks or at a tile change: add its FP32 sums
    // to the registers (and, at a tile change, the registers to P_g) before
    // the next MMA overwrites the accumulator
    const bool run_start = (tile != cur) || run == kTg2Run;
    if (run_start && c > 0) {
      const int pb2 = (c - 1) & 1;
      if (pend[pb2]) {
        if (!(ok = block_wait(&bars[pb2], par[pb2]))) break;
        pend[pb2] = false;
      }
      tc_fence_after();
      tg2_fold(tm_row, tm_acc, acc_first);
      acc_first = false;
      if (tile != cur) {
        tg2_flush(g, cpairs, npairs, cur / n_ntiles, cur - (cur / n_ntiles) * n_ntiles, tm_acc, P);
        acc_first = true;
      }
    }
    if (run_start) run = 0;
    ++run;
    cur = tile;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t ah = umma_desc(Ah + ks * 128, 128, sbo), al = umma_desc(Al + ks * 128, 128, sbo);
        const uint64_t bh = umma_desc(Bh + ks * 128, 128, sbo), bl = umma_desc(Bl + ks * 128, 128, sbo);
        mma_f16(tmem, ah, bh, idesc, (!run_start || ks > 0) ? 1u : 0u);
        mma_f16(tmem, ah, bl, idesc, 1u);
        mma_f16(tmem, al, bh, idesc, 1u);
      }
      mma_commit(&bars[buf]);
    }
    pend[buf] = true;
  }
  // drain: the most recent commit covers every MMA issued before it (after a
  // timeout the accumulator is not read, only waited for before TMEM is freed)
  if (c > 0) {
    const int lb = (c - 1) & 1;
    if (pend[lb] && !block_wait(&bars[lb], par[lb])) ok = false;
  }
  if (!ok) {
    if (tid == 0) atomicExch(status, (int)kDevTimeout);
  } else if (cur >= 0) {
    tc_fence_after();
    tg2_fold(tm_row, tm_acc, acc_first);
    tg2_flush(g, cpairs, npairs, cur / n_ntiles, cur - (cur / n_ntiles) * n_ntiles, tm_acc, P);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

size_t tc_gram2_smem(const Geo& g) {
  return sizeof(uint16_t) * 2 * (2 * kTg2ImgA + 2 * kTg2ImgB) +
         sizeof(float2) * (size_t)tg2_groups_per_tile(g.w) * g.w * kTg2PS + 16 + sizeof(int4) * kTg2KC + 64;
}

cudaError_t launch_tc_gram2(const Geo& g, const float2* chat, const int* pix, const int* dK, int Kpad,
                            const int* pref, const int2* cpairs, int npairs, double2* P, int* status,
                            cudaStream_t st) {
  const size_t sm = tc_gram2_smem(g);
  static size_t attr = 0;
  if (sm > attr) {
    cudaFuncSetAttribute(k_tc_gram2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  const int n_mtiles = (npairs + 127) / 128;
  const int n_ntiles = (g.G * g.w * g.w + 127) / 128;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  note_launches(1);
  k_tc_gram2<<<nsm, kTg2Threads, sm, st>>>(g, chat, pix, dK, Kpad, pref, cpairs, npairs, n_mtiles * n_ntiles,
                                           n_ntiles, P, status);
  return cudaGetLastError();
}

}  // namespace gpjc
