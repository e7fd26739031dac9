// Readout stage of E_c, FP32 register-tiled kernel, and the host tables of
// the register tiles of both readout directions (Eq. 13-15).
#include "k_readout.cuh"

namespace gpjc {

// ------------------------------------------------------------------ host side --
static int ceil_div(int a, int b) { return (a + b - 1) / b; }

size_t readout_fwd_smem(const Geo& g, int rb) {
  const int st = u_stride(g.ntx);
  return sizeof(float2) * (size_t)(upad_size(rb * st) + 2 * spad_size(g.ntx) + g.nx);
}

size_t readout_adj_smem(const Geo& g, int rb, int hstage) {
  const int st = u_stride(g.ntx);
  return sizeof(float2) *
         (size_t)(spad_size(rb * st) + spad_size(g.ntx) + g.nx + (hstage ? 1 + std::max(hpad_size(rb * g.ntxc), hswz_size(rb * g.ntxc)) : 0));
}

size_t readout_fwd2_smem(const Geo& g, int rb, int nb) {
  return sizeof(float2) * ((size_t)nb * fwd2_usz(rb, g.ntx) + (size_t)nb * rb * (g.nx + g.ntx) + g.nx);
}

void build_readout_tiles(const ReadoutGeomHost& h, int rb, bool adjoint, int ts, std::vector<int4>* hdr,
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
    const int step = adjoint ? ts : 4;
    for (int i0 = 0; i0 < inner; i0 += step) {
      for (int c0 = 0; c0 < ncol; c0 += 4) {
        hdr->push_back(make_int4(h.aoff[g] + i0, h.keep[g], std::min(step, inner - i0), 0));
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

double readout_col_fill(const ReadoutGeomHost& h, int rb, bool adjoint, int ts) {
  std::vector<int> occ(h.G, 0);
  for (int p = 0; p < (int)h.pg.size(); ++p) ++occ[h.pg[p]];
  double useful = 0.0, total = 0.0;
  for (int g = 0; g < h.G; ++g) {
    const int kb = ceil_div(adjoint ? h.w : h.keep[g], adjoint ? ts : 4);
    useful += (double)kb * rb * occ[g];
    total += (double)kb * 4 * ceil_div(rb * occ[g], 4);
  }
  return total > 0.0 ? useful / total : 1.0;
}

int readout_tile_count(const ReadoutGeomHost& h, int rb, bool adjoint, int ts) {
  std::vector<std::vector<int>> occ(h.G);
  for (int p = 0; p < (int)h.pg.size(); ++p) occ[h.pg[p]].push_back(p);
  int n = 0;
  for (int g = 0; g < h.G; ++g)
    n += ceil_div(adjoint ? h.w : h.keep[g], adjoint ? ts : 4) * ceil_div(rb * (int)occ[g].size(), 4);
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
    cudaFuncSetAttribute(k1f_tiled<MAXT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         readout_carveout((const void*)k1f_tiled<MAXT>, sm));
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

}  // namespace gpjc
