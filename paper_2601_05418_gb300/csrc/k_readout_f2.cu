// Readout stage of E_c, FP32 register-tiled kernel with batched readout
// transforms (several coils and all rows of a block per two-pass FFT call;
// Eq. 13-15).
#include "k_readout.cuh"

namespace gpjc {

template <int MAXT>
static size_t prepare_fb(const Geo& g, const RTiles& tl) {
  const size_t sm = readout_fwd2_smem(g, tl.rb, tl.nb);
  static int attr = 0;
  if ((int)sm > attr) {
    cudaFuncSetAttribute(k1f_batched<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k1f_batched<MAXT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         readout_carveout((const void*)k1f_batched<MAXT>, sm));
    attr = (int)sm;
  }
  return sm;
}

template <int MAXT>
static cudaError_t launch_fb(const Geo& g, const RTiles& tl, const float2* x, const float2* coil, const float2* AT,
                             float2* Hpart, int nchunk, bool balanced, cudaStream_t st) {
  const size_t sm = prepare_fb<MAXT>(g, tl);
  note_launches(1);
  if (balanced) {
    k1f_batched<MAXT><<<tl.bal_grid, kRThreads, sm, st>>>(g, tl, x, coil, AT, Hpart, 0, tl.nb, tl.bal_units,
                                                          tl.bal_npair, tl.bal_planes);
  } else {
    const int cpc = (g.nc + nchunk - 1) / nchunk;
    dim3 grid((g.rows + tl.rb - 1) / tl.rb, nchunk);
    k1f_batched<MAXT><<<grid, kRThreads, sm, st>>>(g, tl, x, coil, AT, Hpart, cpc, tl.nb, 0, 0, nchunk);
  }
  return cudaGetLastError();
}

template <int MAXT>
static int resident_fb(const Geo& g, const RTiles& tl) {
  const size_t sm = prepare_fb<MAXT>(g, tl);
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1f_batched<MAXT>, kRThreads, sm) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * nsm;
}

cudaError_t launch_k1f_batched(const Geo& g, const RTiles& tl, const float2* x, const float2* coil,
                               const float2* AT, float2* Hpart, int nchunk, bool balanced, cudaStream_t st) {
  if (g.fx.n1 <= 0 || tl.nb < 1 || tl.nb > kReadoutMaxNb) return cudaErrorInvalidValue;
  if (balanced && (tl.bal_units <= 0 || tl.bal_grid <= 0)) return cudaErrorInvalidValue;
  const int maxt = (tl.nt + kRThreads - 1) / kRThreads;
  if (maxt <= 1) return launch_fb<1>(g, tl, x, coil, AT, Hpart, nchunk, balanced, st);
  if (maxt <= 2) return launch_fb<2>(g, tl, x, coil, AT, Hpart, nchunk, balanced, st);
  if (maxt <= 3) return launch_fb<3>(g, tl, x, coil, AT, Hpart, nchunk, balanced, st);
  return cudaErrorInvalidValue;
}

int k1f_batched_resident(const Geo& g, const RTiles& tl) {
  if (g.fx.n1 <= 0 || tl.nb < 1) return 0;
  const int maxt = (tl.nt + kRThreads - 1) / kRThreads;
  if (maxt <= 1) return resident_fb<1>(g, tl);
  if (maxt <= 2) return resident_fb<2>(g, tl);
  if (maxt <= 3) return resident_fb<3>(g, tl);
  return 0;
}

}  // namespace gpjc
