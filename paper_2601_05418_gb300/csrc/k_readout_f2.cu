// Readout stage of E_c, FP32 register-tiled kernel with batched readout
// transforms (several coils and all rows of a block per two-pass FFT call;
// Eq. 13-15).
#include "k_readout.cuh"

namespace gpjc {

template <int MAXT>
static cudaError_t launch_fb(const Geo& g, const RTiles& tl, const float2* x, const float2* coil, const float2* AT,
                             float2* Hpart, int nchunk, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  const size_t sm = readout_fwd2_smem(g, tl.rb, tl.nb);
  static int attr = 0;
  if ((int)sm > attr) {
    cudaFuncSetAttribute(k1f_batched<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k1f_batched<MAXT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         readout_carveout((const void*)k1f_batched<MAXT>, sm));
    attr = (int)sm;
  }
  dim3 grid((g.rows + tl.rb - 1) / tl.rb, nchunk);
  note_launches(1); k1f_batched<MAXT><<<grid, kRThreads, sm, st>>>(g, tl, x, coil, AT, Hpart, cpc, tl.nb);
  return cudaGetLastError();
}

cudaError_t launch_k1f_batched(const Geo& g, const RTiles& tl, const float2* x, const float2* coil,
                               const float2* AT, float2* Hpart, int nchunk, cudaStream_t st) {
  if (g.fx.n1 <= 0 || tl.nb < 1 || tl.nb > kReadoutMaxNb) return cudaErrorInvalidValue;
  const int maxt = (tl.nt + kRThreads - 1) / kRThreads;
  if (maxt <= 1) return launch_fb<1>(g, tl, x, coil, AT, Hpart, nchunk, st);
  if (maxt <= 2) return launch_fb<2>(g, tl, x, coil, AT, Hpart, nchunk, st);
  if (maxt <= 3) return launch_fb<3>(g, tl, x, coil, AT, Hpart, nchunk, st);
  return cudaErrorInvalidValue;
}

}  // namespace gpjc
