#include "k_readout.cuh"

// ====================================================================== batch --
// Many 2D slices of different sizes and coil counts reconstructed by CG in
// ONE persistent launch.  Every (slice, stage, tile) is a work item; a
// global queue hands items out in the order stage-major, then slice, then
// tile, and each item waits (bounded) until all items of the previous stage
// of the same slice are done.  Stages per slice: E_c^H S' (phase-encode,
// readout adjoint, vector init), then per iteration readout forward,
// phase-encode mask projection with ||E_c p||^2, readout adjoint, and the two
// CG vector updates.  Dependencies only point to earlier queue positions and
// all blocks are co-resident (cooperative launch), so the queue cannot
// deadlock; a wait that exceeds its budget sets the abort flag and every
// block leaves.
namespace gpjc {

constexpr int kVecChunk = 2048;  // vector elements per item

enum BatchStage : int { kBPeAdj = 0, kBAdj = 1, kBInit = 2, kBFwd = 3, kBPeN = 4, kBU1 = 5, kBU2 = 6 };

__device__ __forceinline__ int batch_stage_type(int j) {
  if (j < 3) return j;  // kBPeAdj, kBAdj, kBInit
  const int k = (j - 3) % 5;
  return k == 0 ? kBFwd : k == 1 ? kBPeN : k == 2 ? kBAdj : k == 3 ? kBU1 : kBU2;
}

__device__ __forceinline__ int batch_items(const BatchSlice& s, int type) {
  switch (type) {
    case kBPeAdj:
    case kBPeN: return s.n_pe;
    case kBAdj: return s.n_a;
    case kBFwd: return s.n_f;
    default: return s.n_vec;
  }
}

// Each readout body variant is its own (not inlined) device function, so
// the compiler optimises the variants one by one instead of one huge kernel.
template <int MAXT>
__device__ __noinline__ void batch_fwd_v(const BatchSlice& s, const Geo& g, int rblock, int chunk, float2* sm) {
  k1f_body<MAXT, true>(g, s.rtf, s.p, s.coil, s.AT, s.Hpart, s.cpc, rblock, chunk, sm);
}
template <int MAXX, int TS>
__device__ __noinline__ void batch_adj_v(const BatchSlice& s, const Geo& g, int rblock, int chunk, float2* sm) {
  k1a_body<MAXX, true, TS>(g, s.rta, s.H2, s.coil, s.A, s.xparts, s.cpc, rblock, chunk, sm);
}

template <bool FWD>
__device__ __forceinline__ void batch_readout(const BatchSlice& s, const Geo& g, int li, float2* sm) {
  const int rblock = li / s.nchunk, chunk = li - rblock * s.nchunk;
  if (FWD) {
    if (s.mt_f <= 1)
      batch_fwd_v<1>(s, g, rblock, chunk, sm);
    else
      batch_fwd_v<2>(s, g, rblock, chunk, sm);
  } else {
    switch (s.mx_a) {
      case 1: batch_adj_v<1, 4>(s, g, rblock, chunk, sm); break;
      case 2: batch_adj_v<2, 4>(s, g, rblock, chunk, sm); break;
      case 4: batch_adj_v<4, 4>(s, g, rblock, chunk, sm); break;
      case 5: batch_adj_v<1, 2>(s, g, rblock, chunk, sm); break;
      case 6: batch_adj_v<2, 2>(s, g, rblock, chunk, sm); break;
      default: batch_adj_v<8, 4>(s, g, rblock, chunk, sm); break;
    }
  }
}

__global__ void __launch_bounds__(kRThreads) k_batch_cg(BatchPlan bp) {
  extern __shared__ float2 bsm[];
  __shared__ Geo sg;
  __shared__ long long s_item;
  __shared__ int s_ok;
  __shared__ double red[32];
  const long long total = bp.stage_start[bp.n_stages];
  for (;;) {
    if (threadIdx.x == 0) {
      long long it = (long long)atomicAdd(bp.head, 1ull);
      if (*(volatile int*)bp.abort) it = total;
      s_item = it;
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= total) break;
    // decode (stage j, slice s, local item li)
    int lo = 0, hi = bp.n_stages;  // stage_start[lo] <= item < stage_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (bp.stage_start[mid] <= item) lo = mid; else hi = mid;
    }
    const int j = lo, type = batch_stage_type(j);
    const int* so = bp.slice_off + (size_t)type * (bp.n_slices + 1);
    const int rem = (int)(item - bp.stage_start[j]);
    int a = 0, b = bp.n_slices;
    while (b - a > 1) {
      const int mid = (a + b) >> 1;
      if (so[mid] <= rem) a = mid; else b = mid;
    }
    const int si = a, li = rem - so[a];
    const BatchSlice& S = bp.slices[si];
    // wait for the previous stage of this slice
    if (threadIdx.x == 0) {
      int ok = 1;
      if (j > 0) {
        const int need = batch_items(S, batch_stage_type(j - 1));
        volatile int* d = bp.done + (size_t)si * bp.n_stages + (j - 1);
        const long long t0 = clock64();
        while (*d < need) {
          if (*(volatile int*)bp.abort || clock64() - t0 > bp.wait_cycles) {
            ok = 0;
            atomicExch(bp.abort, 1);
            atomicExch(bp.status, (int)kDevTimeout);
            break;
          }
        }
        __threadfence();
      }
      s_ok = ok;
    }
    // slice geometry into shared memory
    {
      const int* src = reinterpret_cast<const int*>(&S.g);
      int* dst = reinterpret_cast<int*>(&sg);
      for (int i = threadIdx.x; i < (int)(sizeof(Geo) / sizeof(int)); i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    if (!s_ok) break;
    const Geo& g = sg;
    const int iter = j < 3 ? -1 : (j - 3) / 5;
    const size_t L = (size_t)g.rows * g.nx;
    switch (type) {
      case kBPeAdj: pe_adj2d_body(g, S.Sc, g.ntxc, S.H2, li, bsm); break;
      case kBAdj: batch_readout<false>(S, g, li, bsm); break;
      case kBFwd: batch_readout<true>(S, g, li, bsm); break;
      case kBPeN: {
        const double tot = pe_normal2d_body<true>(g, S.Hpart, S.nchunk, g.ntxc, S.H2, li, bsm);
        if (threadIdx.x == 0) atomicAdd(S.qq + iter, tot);
        break;
      }
      case kBInit:
      case kBU1: {
        double alpha = 0.0;
        if (type == kBU1) {
          const double rr = __ldcg(S.rr + iter), qq = __ldcg(S.qq + iter);
          alpha = rr == 0.0 ? 0.0 : rr / qq;
          if (!isfinite(alpha)) {
            if (threadIdx.x == 0) atomicExch(bp.status, (int)kDevNonFinite);
            alpha = 0.0;
          }
        }
        const float af = (float)alpha;
        double part = 0.0;
        const size_t i0 = (size_t)li * kVecChunk, i1 = min(L, i0 + kVecChunk);
        for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
          float2 v = __ldcg(S.xparts + i);
          for (int c = 1; c < S.nchunk; ++c) v = cadd(v, __ldcg(S.xparts + c * L + i));
          if (type == kBInit) {  // b = E_c^H S'; x = 0; r = p = b
            S.x[i] = make_float2(0.f, 0.f);
            S.r[i] = v;
            S.p[i] = v;
            part += (double)v.x * v.x + (double)v.y * v.y;
          } else {
            const float2 pv = __ldcg(S.p + i);
            float2 xv = __ldcg(S.x + i), rv = __ldcg(S.r + i);
            xv.x = fmaf(af, pv.x, xv.x);
            xv.y = fmaf(af, pv.y, xv.y);
            rv.x = fmaf(-af, v.x, rv.x);
            rv.y = fmaf(-af, v.y, rv.y);
            S.x[i] = xv;
            S.r[i] = rv;
            part += (double)rv.x * rv.x + (double)rv.y * rv.y;
          }
        }
        const double tot = block_sum(part, red);
        if (threadIdx.x == 0) atomicAdd(S.rr + (type == kBInit ? 0 : iter + 1), tot);
        break;
      }
      case kBU2: {
        const double rr = __ldcg(S.rr + iter), rn = __ldcg(S.rr + iter + 1);
        double beta = rr == 0.0 ? 0.0 : rn / rr;
        if (!isfinite(beta)) beta = 0.0;
        const float bf = (float)beta;
        const size_t i0 = (size_t)li * kVecChunk, i1 = min(L, i0 + kVecChunk);
        if (rr != 0.0)
          for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const float2 rv = __ldcg(S.r + i);
            float2 pv = __ldcg(S.p + i);
            pv.x = fmaf(bf, pv.x, rv.x);
            pv.y = fmaf(bf, pv.y, rv.y);
            S.p[i] = pv;
          }
        break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(bp.done + (size_t)si * bp.n_stages + j, 1);
    }
  }
}

size_t batch_pe_smem(const Geo& g) { return sizeof(float2) * (size_t)(2 * kPeCB * (g.ny + 1) + g.ny); }

cudaError_t launch_batch_cg(const BatchPlan& bp, int grid, size_t smem, cudaStream_t st) {
  static size_t attr = 0;
  if (smem > attr) {
    cudaFuncSetAttribute(k_batch_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_batch_cg, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kRThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launches(1);
  return cudaLaunchKernelEx(&cfg, k_batch_cg, bp);
}

int batch_max_blocks(size_t smem) {
  cudaFuncSetAttribute(k_batch_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, nsm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_cg, kRThreads, smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace gpjc
