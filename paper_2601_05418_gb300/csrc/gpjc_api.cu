// Host side of the C ABI declared in include/gpjc.h: validation, the
// bookkeeping of Sec. 2.3-2.4 (patch offsets, compressed readout length
// N'_tx = sum_p keep[g(p)] of Eq. 15, first patch of each group), handle
// lifetimes, workspaces and the launch sequences of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gpjc.h"
#include "gpjc_internal.h"
#include "gpjc_kernels.h"

using namespace gpjc;

static constexpr int kVecChunkHost = 2048;  // vector elements per batch work item (k_readout.cu)
static constexpr int kPeCBHost = 8;  // columns per phase-encode block (kPeCB)

// ------------------------------------------------------------------ launches --
#include <atomic>
static std::atomic<unsigned long long> g_launches{0};
static thread_local bool g_capturing = false;
namespace gpjc {
void note_launches(int n) {
  if (!g_capturing) g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}
}  // namespace gpjc
extern "C" uint64_t gpjc_launch_count(void) { return g_launches.load(); }

// ------------------------------------------------------------------ errors --
static thread_local std::string g_err;

static gpjc_status fail(gpjc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(GPJC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char* gpjc_strerror(gpjc_status s) {
  switch (s) {
    case GPJC_OK: return "ok";
    case GPJC_EINVAL: return "invalid argument";
    case GPJC_ENOMEM: return "out of memory";
    case GPJC_ECUDA: return "CUDA error";
    case GPJC_ETIMEOUT: return "device wait timed out";
    case GPJC_ENONFINITE: return "non-finite value in reconstruction";
    case GPJC_EUNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}
extern "C" const char* gpjc_last_error(void) { return g_err.c_str(); }
extern "C" const char* gpjc_version(void) { return "gpjc 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ memory --
// Allocation-failure injection for tests of the out-of-memory paths: after
// gpjc_debug_fail_allocations(n), the (n+1)-th and later device allocations
// of the library fail with GPJC_ENOMEM without calling cudaMalloc (n < 0:
// off).  Process-wide.
static std::atomic<long long> g_alloc_budget{-1};
static bool alloc_refused() {
  long long b = g_alloc_budget.load();
  while (b >= 0) {
    if (b == 0) return true;
    if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return false;
  }
  return false;
}
extern "C" void gpjc_debug_fail_allocations(int64_t n) { g_alloc_budget.store(n < 0 ? -1 : n); }

namespace {

struct DevMem {
  std::vector<void*> ptrs;
  ~DevMem() { release(); }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
  template <typename T>
  gpjc_status alloc(T** out, size_t n) {
    *out = nullptr;
    if (n == 0) n = 1;
    if (alloc_refused()) return fail(GPJC_ENOMEM, "cudaMalloc(%zu bytes): refused (injected)", n * sizeof(T));
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(GPJC_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    *out = (T*)p;
    return GPJC_OK;
  }
  template <typename T>
  gpjc_status upload(T** out, const std::vector<T>& v) {
    gpjc_status s = alloc(out, v.size());
    if (s) return s;
    if (!v.empty()) {
      cudaError_t e = cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return fail(GPJC_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    return GPJC_OK;
  }
};

bool factor_fft(int n, FftPlan* pl) {
  pl->n = n;
  pl->nst = 0;
  pl->n1 = pl->n2 = 0;
  if (n == 1) return true;
  int m = n;
  std::vector<int> r;
  while (m % 8 == 0) { r.push_back(8); m /= 8; }
  while (m % 4 == 0) { r.push_back(4); m /= 4; }
  while (m % 2 == 0) { r.push_back(2); m /= 2; }
  while (m % 7 == 0) { r.push_back(7); m /= 7; }
  while (m % 5 == 0) { r.push_back(5); m /= 5; }
  while (m % 3 == 0) { r.push_back(3); m /= 3; }
  if (m != 1 || (int)r.size() > kMaxStages) return false;
  pl->nst = (int)r.size();
  for (int i = 0; i < pl->nst; ++i) pl->rad[i] = r[i];
  pl->n1 = pl->n2 = 0;
  for (int n1 : {16, 8})
    if (n % n1 == 0 && fft2p_supported(n1, n / n1)) {
      pl->n1 = n1;
      pl->n2 = n / n1;
      break;
    }
  return true;
}

}  // namespace

// ------------------------------------------------------------------ plan --
struct gpjc_plan {
  int nx, ny, nz, nc, os, ntx, w, G, np, ns, ntxc, n_lines, keep_max;
  double cycles, kappa_y, kappa_z;
  std::vector<int> pg, keep, poff, ref, aoff, line_ky, line_kz, line_of;
  std::vector<int> out_tbase, out_abase, out_astride;
  Geo geo;
  RTiles rt_f, rt_a;  // register-tiled readout stage (rb == 0: use the per-output kernels)
  bool tc_ok;          // tensor-core compression available (periodic group map, sizes in range)
  // tensor-core geometries: BF16 with FP32 sources (raw data and the BF16
  // operator's spectra; split operands), FP16 with FP32 sources (raw data),
  // FP16 with FP16 sources (the FP16 operator's spectra).  The two FP16 ones
  // share their K chunking, so each format has one set of packed A_g images.
  TcGeom tc32b, tc32h, tc16;
  // aliased sets of the mask (hybrid-space reconstruction, Sec. 3.4): set of
  // each phase-encode row (raster z, y), sets numbered by their first row;
  // CSR member lists (rows ascending) on the host and the device
  int n_sets;
  std::vector<int> set_of_row, set_ptr, set_rows;
  int *d_set_of_row, *d_set_ptr, *d_set_rows;
  DevMem mem;
};

// Aliased sets of a phase-encode mask: the connected components of the
// nonzero pattern of U = F^H M^T M F (F the centred unitary phase-encode DFT,
// M the line selection), |U| > 1e-9 max |U|.  U[r, r''] depends only on the
// row difference: U = c(y - y'', z - z'') / (N_y N_z) with the mask's
// autocorrelation c(dy, dz) = sum_lines exp(2 pi i (ky_c dy / N_y +
// kz_c dz / N_z)), computed as a per-kz sum over the lines followed by a
// DFT over kz.  The components of this circulant pattern are the cosets of
// the subgroup of Z_Ny x Z_Nz that the nonzero differences generate: a
// union-find pass over all rows is needed only for a difference not yet in
// that subgroup (each such pass at least doubles it).
static void aliased_sets(int ny, int nz, const std::vector<int>& ky, const std::vector<int>& kz, int* n_sets,
                         std::vector<int>* set_of_row, std::vector<int>* set_ptr, std::vector<int>* set_rows) {
  const int rows = ny * nz;
  const int nl = (int)ky.size();
  // A[kz][dy] = sum_{lines with this kz} exp(2 pi i ky_c dy / N_y)
  std::vector<std::complex<double>> A((size_t)nz * ny, 0.0);
  for (int l = 0; l < nl; ++l) {
    const double kyc = (double)(ky[l] - ny / 2);
    std::complex<double>* a = &A[(size_t)kz[l] * ny];
    for (int dy = 0; dy < ny; ++dy) {
      const double ph = 2.0 * M_PI * std::fmod(kyc * dy, (double)ny) / ny;
      a[dy] += std::complex<double>(std::cos(ph), std::sin(ph));
    }
  }
  // c(dy, dz) = sum_kz exp(2 pi i kz_c dz / N_z) A[kz][dy]
  std::vector<double> mag((size_t)nz * ny, 0.0);
  for (int dz = 0; dz < nz; ++dz)
    for (int dy = 0; dy < ny; ++dy) {
      std::complex<double> c = 0.0;
      for (int k = 0; k < nz; ++k) {
        const double ph = 2.0 * M_PI * std::fmod((double)(k - nz / 2) * dz, (double)nz) / nz;
        c += std::complex<double>(std::cos(ph), std::sin(ph)) * A[(size_t)k * ny + dy];
      }
      mag[(size_t)dz * ny + dy] = std::abs(c);
    }
  const double thr = 1e-9 * mag[0];  // |c(0)| = number of lines = max |c|
  std::vector<int> parent(rows);
  for (int r = 0; r < rows; ++r) parent[r] = r;
  auto find = [&](int a) {
    while (parent[a] != a) {
      parent[a] = parent[parent[a]];
      a = parent[a];
    }
    return a;
  };
  for (int dz = 0; dz < nz; ++dz)
    for (int dy = 0; dy < ny; ++dy) {
      const int d = dz * ny + dy;
      if (d == 0 || !(mag[d] > thr)) continue;
      if (find(0) == find(d)) continue;  // already in the generated subgroup
      for (int r = 0; r < rows; ++r) {
        const int y = r % ny, z = r / ny;
        const int q = ((z + dz) % nz) * ny + (y + dy) % ny;
        const int a = find(r), b = find(q);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
      }
    }
  // number the sets by their first row
  std::vector<int> id(rows, -1);
  set_of_row->assign(rows, 0);
  int ns = 0;
  for (int r = 0; r < rows; ++r) {
    const int root = find(r);
    if (id[root] < 0) id[root] = ns++;
    (*set_of_row)[r] = id[root];
  }
  set_ptr->assign(ns + 1, 0);
  for (int r = 0; r < rows; ++r) ++(*set_ptr)[(*set_of_row)[r] + 1];
  for (int k = 0; k < ns; ++k) (*set_ptr)[k + 1] += (*set_ptr)[k];
  set_rows->assign(rows, 0);
  std::vector<int> fill(set_ptr->begin(), set_ptr->end() - 1);
  for (int r = 0; r < rows; ++r) (*set_rows)[fill[(*set_of_row)[r]]++] = r;
  *n_sets = ns;
}

// Tensor-core compression geometry for sources of `ebytes` bytes per real
// element; false when the group map or the sizes do not fit the kernels.
static bool make_tc_geom(const gpjc_plan* p, int ebytes, int fmt, TcGeom* t) {
  memset(t, 0, sizeof *t);
  const int G = p->G, w = p->w;
  const long long P = (long long)G * w;
  if (p->ntx % P) return false;
  for (int q = 0; q < p->np; ++q)
    if (p->pg[q] != q % G) return false;
  const int n_occ = (int)(p->ntx / P);
  // a tile holds lt = floor(128 / n_occ) lines; its last 128 - lt n_occ MMA
  // rows are padding
  if (n_occ > 128) return false;
  if (p->keep_max > 128 || w > 64) return false;
  if (((long long)P * ebytes) % 8 || ((long long)p->ntx * ebytes) % 8) return false;
  t->G = G; t->w = w; t->nc = p->nc; t->ns = p->ns; t->ntx = p->ntx; t->ntxc = p->ntxc;
  t->n_occ = n_occ; t->P = (int)P; t->lt = 128 / n_occ;
  int c0 = 1;
  while ((2 * w * c0) % 16) ++c0;
  int ncc = c0;
  // K chunks of at most 64 for FP16, 32 for the split BF16 GEMM (unless one
  // chunk of c0 coils is longer): a block's staging and operand images stay
  // small, so several blocks share an SM and one block's TMA load overlaps
  // the others' conversion and MMAs (2d256 BF16 forward: K chunks of
  // 128 / 64 / 32: 197 / 158 / 146 us; FP16: 132 / 121 / 127 us)
  int kmax = fmt == 1 ? 32 : 64;  // GPJC_TC_KMAX (16..256) overrides the K chunk cap
  if (const char* e = getenv("GPJC_TC_KMAX")) {
    const int v = atoi(e);
    if (v >= 16 && v <= 256) kmax = v;
  }
  while (ncc + c0 <= p->nc && 2 * w * (ncc + c0) <= kmax) ncc += c0;
  t->ncc = ncc;
  t->nchunks = (p->nc + ncc - 1) / ncc;
  t->Kc = 2 * w * ncc;
  t->npad = ((2 * p->keep_max + 15) / 16) * 16;
  t->xalign = 16 / ebytes;
  t->box0 = ((2 * w + t->xalign - 2 + t->xalign - 1) / t->xalign) * t->xalign;
  t->stg_tx = t->box0 * n_occ * ncc * t->lt * ebytes;
  t->stg_bytes = ((t->stg_tx + 1023) / 1024) * 1024;
  int tc = 32;
  while (tc < t->npad) tc *= 2;
  t->tmem_cols = tc;
  t->Kx = ((2 * p->keep_max + 15) / 16) * 16;
  t->nexp = ((2 * p->ns + 15) / 16) * 16;
  if (t->box0 > 256 || ncc > 256 || t->lt > 256 || n_occ > 256) return false;
  if (tc_compress_smem(*t, fmt) > 220 * 1024 || tc_expand_smem(*t, fmt) > 220 * 1024) return false;
  return true;
}

// Coils per step of the batched-transform forward readout kernel
// (k1f_batched): the nb in 1..4 whose two FFT passes (nb rb os N2 and
// nb rb os N1 tasks) keep the largest share of the block's 256 threads busy
// per round, among those whose shared memory leaves room for two blocks per
// SM (the kernel's registers allow two); the smaller nb on ties.  0 keeps the
// per-row kernel (lengths without a two-pass plan, or nothing fits).
// GPJC_READOUT_NB (0..4) overrides.  On the 256 x 256, 32-coil workload nb = 2
// (one row, 16 transforms) took the forward stage from 179 to 157 us; on the
// 224 x 224 x 160 volume nb = 1 with the block's 2 or 4 rows batched saved
// 13-15%.  (The adjoint keeps its per-row kernel: a batched version with the
// second pass in place in the FFT scratch measured 6-20% slower there.)
static int pick_readout_nb(const Geo& g, const RTiles& rt) {
  if (g.fx.n1 <= 0 || rt.rb <= 0) return 0;
  if (const char* e = getenv("GPJC_READOUT_NB")) {
    const int v = atoi(e);
    if (v == 0) return 0;
    if (v >= 1 && v <= kReadoutMaxNb && readout_fwd2_smem(g, rt.rb, v) <= 227 * 1024) return v;
  }
  int best = 0;
  double best_eff = -1.0;
  for (int nb = 1; nb <= std::min(kReadoutMaxNb, g.nc); ++nb) {
    if (readout_fwd2_smem(g, rt.rb, nb) > 112 * 1024) break;
    const long t1 = (long)nb * rt.rb * g.os * g.fx.n2, t2 = (long)nb * rt.rb * g.os * g.fx.n1;
    const double eff = double(t1 + t2) / (256.0 * double((t1 + 255) / 256 + (t2 + 255) / 256));
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = nb;
    }
  }
  return best;
}

// Balanced launch of the batched forward readout (k1f_batched): one wave of
// the device's resident blocks over (row block, group of nb coils) units, so
// no wave runs partly empty (2d256: 256 row blocks on 304 resident blocks
// leave 48 SMs with one block where the others have two: forward stage 164 ->
// 151 us, with the phase-encode stage reading 3 planes instead of 1).  Used
// when the row blocks make fewer than 4 waves of resident blocks (with more,
// the last wave's idle share is small and the extra planes cost more: the
// 224 x 224 x 160 volume's 17920 row blocks ran 2% slower balanced) and every
// block gets at least two units; the planes a row block's segments need are
// bounded by 2 + (units per row block - 1) / (fewest units per block), since
// block boundaries are at least that many units apart.  GPJC_READOUT_BALANCE=0
// keeps the row-block x coil-chunk grid.
static void pick_readout_balance(const Geo& g, RTiles* rt) {
  if (const char* e = getenv("GPJC_READOUT_BALANCE"))
    if (e[0] == '0') return;
  const int grid = k1f_batched_resident(g, *rt);
  const int npair = (g.nc + rt->nb - 1) / rt->nb;
  const long long rblocks = (g.rows + rt->rb - 1) / rt->rb, units = rblocks * npair;
  if (grid <= 0 || rblocks >= 4LL * grid || units < 2LL * grid || units > (1LL << 30)) return;
  const int minblk = (int)(units / grid);
  rt->bal_grid = grid;
  rt->bal_units = (int)units;
  rt->bal_npair = npair;
  rt->bal_planes = 2 + (npair - 1) / minblk;
}

extern "C" gpjc_status gpjc_plan_create(const gpjc_geom* gm, gpjc_plan** out) {
  if (!gm || !out) return fail(GPJC_EINVAL, "null geometry or output pointer");
  *out = nullptr;
  const int nx = gm->nx, ny = gm->ny, nz = gm->nz, nc = gm->nc, os = gm->os, w = gm->w, G = gm->n_groups;
  if (nx < 2 || ny < 2 || (nx & 1) || (ny & 1)) return fail(GPJC_EINVAL, "nx, ny must be even and >= 2");
  if (nz < 1 || (nz > 1 && (nz & 1))) return fail(GPJC_EINVAL, "nz must be 1 or even");
  if (nc < 1 || nc > 64) return fail(GPJC_EINVAL, "nc must be in [1, 64]");
  if (os < 1 || os > 16) return fail(GPJC_EINVAL, "os must be in [1, 16]");
  const long long ntx = (long long)os * nx;
  if (w < 1 || ntx % w) return fail(GPJC_EINVAL, "w must divide ntx = os*nx");
  if (G < 1) return fail(GPJC_EINVAL, "n_groups must be >= 1");
  if (!gm->patch_group || !gm->keep) return fail(GPJC_EINVAL, "patch_group and keep are required");
  if (gm->n_lines < 1 || !gm->line_ky) return fail(GPJC_EINVAL, "at least one sampled line is required");
  if (!std::isfinite(gm->cycles) || !std::isfinite(gm->kappa_y) || !std::isfinite(gm->kappa_z))
    return fail(GPJC_EINVAL, "wave parameters must be finite");
  FftPlan fx, fy, fz;
  if (!factor_fft(nx, &fx) || !factor_fft(ny, &fy) || !factor_fft(nz, &fz))
    return fail(GPJC_EINVAL, "nx, ny, nz must be products of 2, 3, 5, 7");
  auto* p = new (std::nothrow) gpjc_plan();
  if (!p) return fail(GPJC_ENOMEM, "host allocation");
  std::unique_ptr<gpjc_plan> guard(p);
  p->nx = nx; p->ny = ny; p->nz = nz; p->nc = nc; p->os = os; p->ntx = (int)ntx; p->w = w; p->G = G;
  p->np = (int)(ntx / w);
  p->ns = nc * w;
  p->cycles = gm->cycles; p->kappa_y = gm->kappa_y; p->kappa_z = gm->kappa_z;
  p->pg.assign(gm->patch_group, gm->patch_group + p->np);
  p->keep.assign(gm->keep, gm->keep + G);
  std::vector<int> used(G, 0);
  for (int q = 0; q < p->np; ++q) {
    const int g = p->pg[q];
    if (g < 0 || g >= G) return fail(GPJC_EINVAL, "patch_group[%d] = %d out of range", q, g);
    used[g] = 1;
  }
  p->keep_max = 0;
  for (int g = 0; g < G; ++g) {
    if (!used[g]) return fail(GPJC_EINVAL, "group %d has no patch", g);
    if (p->keep[g] < 1 || p->keep[g] > p->ns) return fail(GPJC_EINVAL, "keep[%d] = %d not in [1, N_s]", g, p->keep[g]);
    p->keep_max = std::max(p->keep_max, p->keep[g]);
  }
  // offsets, compressed length, first patch of each group
  p->poff.resize(p->np);
  p->ref.assign(G, -1);
  long long acc = 0;
  for (int q = 0; q < p->np; ++q) {
    p->poff[q] = (int)acc;
    acc += p->keep[p->pg[q]];
    if (p->ref[p->pg[q]] < 0) p->ref[p->pg[q]] = q;
  }
  if (acc > (1 << 24)) return fail(GPJC_EUNSUPPORTED, "compressed readout too long");
  p->ntxc = (int)acc;
  p->aoff.resize(G);
  long long ao = 0;
  for (int g = 0; g < G; ++g) {
    p->aoff[g] = (int)ao;
    ao += (long long)p->ns * p->keep[g];
  }
  if (ao > (1LL << 30)) return fail(GPJC_EUNSUPPORTED, "compression matrices too large");
  p->out_tbase.resize(p->ntxc);
  p->out_abase.resize(p->ntxc);
  p->out_astride.resize(p->ntxc);
  for (int q = 0; q < p->np; ++q) {
    const int g = p->pg[q];
    for (int k = 0; k < p->keep[g]; ++k) {
      const int o = p->poff[q] + k;
      p->out_tbase[o] = q * w;
      p->out_abase[o] = p->aoff[g] + k;
      p->out_astride[o] = p->keep[g];
    }
  }
  // lines
  p->n_lines = gm->n_lines;
  p->line_ky.assign(gm->line_ky, gm->line_ky + gm->n_lines);
  if (gm->line_kz)
    p->line_kz.assign(gm->line_kz, gm->line_kz + gm->n_lines);
  else
    p->line_kz.assign(gm->n_lines, 0);
  p->line_of.assign((size_t)nz * ny, -1);
  for (int l = 0; l < p->n_lines; ++l) {
    const int ky = p->line_ky[l], kz = p->line_kz[l];
    if (ky < 0 || ky >= ny || kz < 0 || kz >= nz) return fail(GPJC_EINVAL, "line %d = (%d, %d) outside the grid", l, kz, ky);
    if (l > 0) {
      const long long prev = (long long)p->line_kz[l - 1] * ny + p->line_ky[l - 1];
      const long long cur = (long long)kz * ny + ky;
      if (cur <= prev) return fail(GPJC_EINVAL, "lines must be unique and sorted by (kz, ky) (line %d)", l);
    }
    p->line_of[(size_t)kz * ny + ky] = l;
  }
  // resource limits of this build
  Geo& g = p->geo;
  memset(&g, 0, sizeof g);
  g.nx = nx; g.ny = ny; g.nz = nz; g.nc = nc; g.os = os; g.ntx = (int)ntx; g.w = w; g.G = G; g.ns = p->ns;
  g.np = p->np; g.ntxc = p->ntxc; g.rows = ny * nz; g.n_lines = p->n_lines; g.keep_max = p->keep_max;
  g.dim3d = nz > 1;
  g.inv_sqrt_ntx = (float)(1.0 / std::sqrt((double)ntx));
  g.inv_sqrt_ny = (float)(1.0 / std::sqrt((double)ny));
  g.inv_sqrt_nz = (float)(1.0 / std::sqrt((double)nz));
  g.fx = fx; g.fy = fy; g.fz = fz;
  const size_t k1adj = k1_smem_bytes(g) + sizeof(float2) * (size_t)g.ntxc;
  if (k1adj > 220 * 1024) return fail(GPJC_EUNSUPPORTED, "readout too long for the shared-memory readout stage");
  if (g.ntxc > 32 * 256) return fail(GPJC_EUNSUPPORTED, "compressed readout longer than 8192");
  if (nx > 512) return fail(GPJC_EUNSUPPORTED, "nx > 512");
  if (ny > 2048 || nz > 2048) return fail(GPJC_EUNSUPPORTED, "phase-encode size > 2048");
  if (w > 64) return fail(GPJC_EUNSUPPORTED, "w > 64");
  // device tables
  DevMem& m = p->mem;
  int *d_pg, *d_poff, *d_keep, *d_aoff, *d_tb, *d_ab, *d_as, *d_ky, *d_kz, *d_lof;
  gpjc_status s;
  if ((s = m.upload(&d_pg, p->pg)) || (s = m.upload(&d_poff, p->poff)) || (s = m.upload(&d_keep, p->keep)) ||
      (s = m.upload(&d_aoff, p->aoff)) || (s = m.upload(&d_tb, p->out_tbase)) ||
      (s = m.upload(&d_ab, p->out_abase)) || (s = m.upload(&d_as, p->out_astride)) ||
      (s = m.upload(&d_ky, p->line_ky)) || (s = m.upload(&d_kz, p->line_kz)) ||
      (s = m.upload(&d_lof, p->line_of)))
    return s;
  float2 *tw_x, *tw_y, *tw_z, *pre, *post_y, *post_z;
  float *ay, *az;
  if ((s = m.alloc(&tw_x, nx)) || (s = m.alloc(&tw_y, ny)) || (s = m.alloc(&tw_z, nz)) ||
      (s = m.alloc(&pre, (size_t)ntx)) || (s = m.alloc(&ay, (size_t)ntx)) || (s = m.alloc(&az, (size_t)ntx)) ||
      (s = m.alloc(&post_y, (size_t)ny * ntx)) || (s = m.alloc(&post_z, (size_t)nz * ntx)))
    return s;
  g.pg = d_pg; g.poff = d_poff; g.keep = d_keep; g.aoff = d_aoff; g.out_tbase = d_tb; g.out_abase = d_ab;
  g.out_astride = d_as; g.line_ky = d_ky; g.line_kz = d_kz; g.line_of = d_lof; g.ay = ay; g.az = az;
  g.tw_x = tw_x; g.tw_y = tw_y; g.tw_z = tw_z; g.pre = pre; g.post_y = post_y; g.post_z = post_z;
  aliased_sets(ny, nz, p->line_ky, p->line_kz, &p->n_sets, &p->set_of_row, &p->set_ptr, &p->set_rows);
  if ((s = m.upload(&p->d_set_of_row, p->set_of_row)) || (s = m.upload(&p->d_set_ptr, p->set_ptr)) ||
      (s = m.upload(&p->d_set_rows, p->set_rows)))
    return s;
  CK(launch_make_tables(g, tw_x, tw_y, tw_z, pre, ay, az, p->cycles, p->kappa_y, p->kappa_z, 0));
  CK(launch_make_post(g, post_y, post_z, p->cycles, p->kappa_y, p->kappa_z, 0));
  p->tc_ok = make_tc_geom(p, 4, 1, &p->tc32b) && make_tc_geom(p, 4, 0, &p->tc32h) && make_tc_geom(p, 2, 0, &p->tc16);
  if (p->tc_ok) {
    for (TcGeom* t : {&p->tc32b, &p->tc32h, &p->tc16}) {
      t->keep = d_keep;
      t->aoff = d_aoff;
      t->poff = d_poff;
    }
  }
  // register-tile tables of the readout stage: the smallest rows-per-block
  // that gives every thread of a block a tile, within the shared-memory and
  // register budgets
  {
    ReadoutGeomHost rh;
    rh.G = G; rh.w = w; rh.ntx = (int)ntx; rh.ntxc = p->ntxc;
    rh.pg = p->pg; rh.keep = p->keep; rh.poff = p->poff; rh.aoff = p->aoff;
    for (int adj = 0; adj < 2; ++adj) {
      int best = 0, ts = 4, hstage = 0;
      // adjoint: one row per block with its row of H2 in shared memory, when
      // that leaves room for three blocks per SM (tiles of 2 samples if 4
      // leave threads without a tile)
      if (adj && readout_adj_smem(g, 1, 1) <= 74 * 1024 && nx <= 512) {
        best = 1;
        hstage = 1;
        ts = readout_tile_count(rh, 1, true, 4) >= 256 ? 4 : 2;
        if ((readout_tile_count(rh, 1, true, ts) + 255) / 256 > 4) best = 0;
      }
      auto fits = [&](int rb) {
        const int nt = readout_tile_count(rh, rb, adj != 0, 4);
        const size_t smem = adj ? readout_adj_smem(g, rb, 0) : readout_fwd_smem(g, rb);
        if (smem > 110 * 1024 || (nt + 255) / 256 > (adj ? 4 : 3) || rb > g.rows) return false;
        return !(adj && (rb * nx + 255) / 256 > 8);
      };
      if (!best) {
        ts = 4;
        hstage = 0;
        for (int rb = 1; rb <= 8; rb *= 2) {
          if (!fits(rb)) break;
          best = rb;
          if (readout_tile_count(rh, rb, adj != 0, 4) >= 256) break;
        }
      }
      // groups with fewer than 4 patches per row (contiguous readout
      // subregions: one) leave most of each 4-column tile empty at one row
      // per block; more rows per block fill the columns (the 224 x 224 x 160
      // volume's 48 contiguous groups: 25% of the contraction's multiply-adds
      // did work at one row, 100% at four)
      if (best && readout_col_fill(rh, best, adj != 0, ts) < 0.75) {
        double f_best = readout_col_fill(rh, best, adj != 0, ts);
        for (int rb = best * 2; rb <= 8; rb *= 2) {
          if (!fits(rb)) break;
          const double f = readout_col_fill(rh, rb, adj != 0, 4);
          if (f > f_best + 1e-9) {
            f_best = f;
            best = rb;
            ts = 4;
            hstage = 0;
          }
        }
      }
      RTiles& rt = adj ? p->rt_a : p->rt_f;
      rt.rb = best;
      rt.nt = 0;
      rt.ts = ts;
      rt.hstage = hstage;
      rt.hdr = nullptr;
      rt.cols = nullptr;
      rt.nb = adj ? 0 : pick_readout_nb(g, rt);
      // paired H2 staging when every patch starts on a 16-component boundary
      // and every group keeps an even count <= 16 (all adjoint tiles of a
      // full column block then read their components in pairs)
      rt.hpair = 0;
      if (adj && hstage) {
        bool ok = true;
        for (size_t q = 0; q < p->pg.size() && ok; ++q) {
          const int kq = p->keep[p->pg[q]];
          ok = (p->poff[q] & 15) == 0 && kq <= 16 && (kq & 1) == 0;
        }
        rt.hpair = ok ? 1 : 0;
      }
      if (best) {
        std::vector<int4> hdr, cols;
        build_readout_tiles(rh, best, adj != 0, ts, &hdr, &cols);
        int4 *dh, *dc;
        if ((s = m.upload(&dh, hdr)) || (s = m.upload(&dc, cols))) return s;
        rt.nt = (int)hdr.size();
        rt.hdr = dh;
        rt.cols = dc;
      }
      rt.bal_grid = rt.bal_units = rt.bal_npair = rt.bal_planes = 0;
      if (!adj && best && rt.nb) pick_readout_balance(g, &rt);
    }
  }
  CK(cudaDeviceSynchronize());
  *out = guard.release();
  return GPJC_OK;
}

extern "C" void gpjc_plan_destroy(gpjc_plan* plan) { delete plan; }

extern "C" gpjc_status gpjc_plan_ntx_c(const gpjc_plan* plan, int32_t* ntx_c) {
  if (!plan || !ntx_c) return fail(GPJC_EINVAL, "null argument");
  *ntx_c = plan->ntxc;
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_plan_sets(const gpjc_plan* plan, int32_t* h_set_of_row, int32_t* n_sets) {
  if (!plan) return fail(GPJC_EINVAL, "null plan");
  if (n_sets) *n_sets = plan->n_sets;
  if (h_set_of_row) std::copy(plan->set_of_row.begin(), plan->set_of_row.end(), h_set_of_row);
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_plan_tables(const gpjc_plan* plan, int32_t* h_off, int32_t* h_ref, int32_t* h_line_of) {
  if (!plan) return fail(GPJC_EINVAL, "null plan");
  if (h_off) std::copy(plan->poff.begin(), plan->poff.end(), h_off);
  if (h_ref) std::copy(plan->ref.begin(), plan->ref.end(), h_ref);
  if (h_line_of) std::copy(plan->line_of.begin(), plan->line_of.end(), h_line_of);
  return GPJC_OK;
}

// ------------------------------------------------------------------ groups --
struct gpjc_groups {
  const gpjc_plan* plan;
  float2* A;        // [aoff[g] + k ns + i]
  float2* AT;       // [aoff[g] + i keep_g + k]
  float* scale;     // [G]
  int* pix;         // [L] (first K used)
  int* dK;          // device |ROI|
  double2* P;       // [G][ns][ns]
  bool built;       // from coil maps (vs. from matrices)
  bool keep_gram;
  int b, iters, iters32, nblk, Kpad;
  float2 *P32, *X32, *Y32;  // FP32 phase of the subspace iteration
  int2* tg_pairs;           // coil pairs (n, n'), n <= n', of the tensor-core Gram
  int tg_npairs;
  bool tc_gram;             // tensor-core Gram (default) or the FFMA one
  // scratch kept for rebuilds, so a rebuild allocates nothing and does
  // not synchronise
  int *blockcount, *blockoff, *d_ref;
  float2 *chat, *dT;
  double2 *X, *Y, *U, *Hm, *W;
  double *ritz, *resid;
  int* order;
  // tensor-core packs of A_g (index 0: FP16, 1: BF16): compression B per
  // (group, coil chunk) and expansion B per group; refreshed on every build
  uint16_t* tc_bc[2];
  uint16_t* tc_bx[2];
  int* tc_status;
  // host copies, read lazily
  mutable bool host_valid;
  mutable long long K;
  mutable std::vector<double> ritz_h;
  mutable double max_resid;
  DevMem mem;
};

static gpjc_status groups_alloc_A(gpjc_groups* gr) {
  const gpjc_plan* p = gr->plan;
  const size_t na = (size_t)p->aoff.back() + (size_t)p->ns * p->keep.back();
  gpjc_status s;
  if ((s = gr->mem.alloc(&gr->A, na)) || (s = gr->mem.alloc(&gr->AT, na)) || (s = gr->mem.alloc(&gr->scale, p->G)))
    return s;
  gr->tc_bc[0] = gr->tc_bc[1] = gr->tc_bx[0] = gr->tc_bx[1] = nullptr;
  gr->tc_status = nullptr;
  if (p->tc_ok) {
    for (int f = 0; f < 2; ++f) {
      const TcGeom& t = f ? p->tc32b : p->tc16;  // the chunking of the format's packs
      if ((s = gr->mem.alloc(&gr->tc_bc[f], tc_pack_comp_elems(t, f))) ||
          (s = gr->mem.alloc(&gr->tc_bx[f], tc_pack_exp_elems(t, f))))
        return s;
    }
    if ((s = gr->mem.alloc(&gr->tc_status, 1))) return s;
    CK(cudaMemset(gr->tc_status, 0, sizeof(int)));
  }
  return GPJC_OK;
}

// re-packs the tensor-core images of A_g after A changed
static gpjc_status groups_pack_tc(gpjc_groups* gr, cudaStream_t st) {
  const gpjc_plan* p = gr->plan;
  if (!p->tc_ok) return GPJC_OK;
  for (int f = 0; f < 2; ++f) {
    // the packs depend only on N, K and the format's chunking
    TcGeom t = f ? p->tc32b : p->tc16;
    t.scale = gr->scale;
    CK(launch_tc_pack(t, f, gr->A, gr->scale, gr->tc_bc[f], gr->tc_bx[f], st));
  }
  return GPJC_OK;
}

// Asynchronous group build on `st` into the scratch of `gr`.
static gpjc_status groups_compute(gpjc_groups* gr, const float2* coil, const uint8_t* roi, const float* h_T,
                                  cudaStream_t st) {
  const gpjc_plan* plan = gr->plan;
  const Geo& g = plan->geo;
  const int b = gr->b;
  if (h_T) CK(cudaMemcpyAsync(gr->dT, h_T, sizeof(float2) * g.nc * g.nc, cudaMemcpyHostToDevice, st));
  CK(launch_roi_count(g, coil, roi, gr->blockcount, gr->nblk, st));
  CK(launch_roi_scan(gr->blockcount, gr->blockoff, gr->nblk, gr->dK, st));
  CK(launch_roi_compact(g, coil, roi, gr->blockoff, gr->pix, gr->nblk, st));
  CK(launch_roi_coils(g, coil, h_T ? gr->dT : nullptr, gr->pix, gr->dK, gr->Kpad, gr->chat, st));
  CK(cudaMemsetAsync(gr->P, 0, sizeof(double2) * (size_t)g.G * g.ns * g.ns, st));
  if (gr->tc_gram)
    CK(launch_tc_gram2(g, gr->chat, gr->pix, gr->dK, gr->Kpad, gr->d_ref, gr->tg_pairs, gr->tg_npairs, gr->P,
                       gr->tc_status, st));
  else
    CK(launch_gram(g, gr->chat, gr->pix, gr->dK, gr->Kpad, gr->d_ref, gr->P, st));
  CK(launch_hermitize(g, gr->P, st));
  double2 *X = gr->X, *Y = gr->Y;
  CK(launch_eig_init(g, b, X, st));
  if (gr->iters32 > 0) {
    // single-precision iterations first (64x the FP64 rate), then FP64 ones
    const size_t nb = (size_t)g.G * g.ns * b;
    CK(launch_to_f32(gr->P, gr->P32, (size_t)g.G * g.ns * g.ns, st));
    CK(launch_to_f32(X, gr->X32, nb, st));
    float2 *X32 = gr->X32, *Y32 = gr->Y32;
    for (int it = 0; it < gr->iters32; ++it) {
      CK(launch_eig_matmul32(g, b, gr->P32, X32, Y32, st));
      CK(launch_eig_orth32(g, b, Y32, st));
      std::swap(X32, Y32);
    }
    CK(launch_to_f64(X32, X, nb, st));
  }
  for (int it = 0; it < gr->iters; ++it) {
    CK(launch_eig_matmul(g, b, gr->P, X, Y, st));
    CK(launch_eig_orth(g, b, Y, st));
    std::swap(X, Y);
  }
  CK(launch_eig_matmul(g, b, gr->P, X, Y, st));           // Z = P Q
  CK(launch_eig_project(g, b, X, Y, gr->Hm, st));         // Q^H P Q
  CK(launch_eig_jacobi(g, b, gr->Hm, gr->W, gr->ritz, gr->order, 60, st));
  CK(launch_eig_rotate(g, b, X, gr->W, gr->order, gr->U, st));  // Ritz vectors U = Q W, descending
  // P U = (P Q) W = Z W: the same rotation of Z (b^2 instead of N_s^2 work per column)
  CK(launch_eig_rotate(g, b, Y, gr->W, gr->order, X, st));
  CK(launch_eig_residual(g, b, X, gr->U, gr->ritz, gr->order, gr->resid, st));
  CK(launch_form_A(g, b, gr->U, h_T ? gr->dT : nullptr, gr->A, gr->AT, gr->scale, st));
  gr->host_valid = false;
  return groups_pack_tc(gr, st);
}

// Reads |ROI|, Ritz values and residuals back (synchronous).
static gpjc_status groups_sync_host(const gpjc_groups* gr) {
  if (gr->host_valid || !gr->built) return GPJC_OK;
  const Geo& g = gr->plan->geo;
  const int b = gr->b;
  int K = 0;
  std::vector<double> rz((size_t)g.G * b), rs(g.G);
  std::vector<int> ord((size_t)g.G * b);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&K, gr->dK, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(rz.data(), gr->ritz, sizeof(double) * rz.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ord.data(), gr->order, sizeof(int) * ord.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(rs.data(), gr->resid, sizeof(double) * rs.size(), cudaMemcpyDeviceToHost));
  gr->K = K;
  gr->ritz_h.resize(rz.size());
  for (int gg = 0; gg < g.G; ++gg)
    for (int r = 0; r < b; ++r) gr->ritz_h[(size_t)gg * b + r] = rz[(size_t)gg * b + ord[(size_t)gg * b + r]];
  gr->max_resid = 0.0;
  for (double v : rs) gr->max_resid = std::max(gr->max_resid, v);
  gr->host_valid = true;
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_build_groups(const gpjc_plan* plan, const float* d_coil, const uint8_t* d_roi,
                                         const float* h_T, const gpjc_build_params* params, void* stream,
                                         gpjc_groups** out) {
  if (!plan || !d_coil || !d_roi || !out) return fail(GPJC_EINVAL, "null argument");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  const Geo& g = plan->geo;
  gpjc_build_params bp = {0, 0, 0, 0};
  if (params) bp = *params;
  if (bp.eig_iters < 0 || bp.eig_iters > 1000) return fail(GPJC_EINVAL, "eig_iters out of range");
  if (bp.eig_iters_fp32 < -1 || bp.eig_iters_fp32 > 1000) return fail(GPJC_EINVAL, "eig_iters_fp32 out of range");
  int b = bp.block;
  if (b <= 0) b = std::min(plan->ns, std::min(96, std::max(2 * plan->keep_max, plan->keep_max + 16)));
  if (b < plan->keep_max || b > plan->ns) return fail(GPJC_EINVAL, "block %d must be in [keep_max, N_s]", b);
  if (b > 96) return fail(GPJC_EUNSUPPORTED, "subspace block > 96 (keep too large)");
  auto* gr = new (std::nothrow) gpjc_groups();
  if (!gr) return fail(GPJC_ENOMEM, "host allocation");
  std::unique_ptr<gpjc_groups> guard(gr);
  gr->plan = plan;
  gr->b = b;
  // six FP32 iterations reach the FP32 rounding floor of the subspace on the
  // slowest-converging workload geometry (3D, lambda_{b+1} / lambda_keep ~ 0.06);
  // more change nothing measurable
  gr->iters32 = bp.eig_iters_fp32 > 0 ? bp.eig_iters_fp32 : (bp.eig_iters_fp32 < 0 ? 0 : 6);
  // after the FP32 phase one FP64 iteration reaches FP64 accuracy (its
  // subspace error is already at the FP32 rounding level); without it the
  // FP64 iteration starts from random vectors
  gr->iters = bp.eig_iters > 0 ? bp.eig_iters : (gr->iters32 > 0 ? 1 : 12);
  gr->keep_gram = bp.keep_gram != 0;
  gr->built = true;
  gr->host_valid = false;
  gpjc_status s;
  if ((s = groups_alloc_A(gr))) return s;
  DevMem& m = gr->mem;
  const size_t L = (size_t)g.rows * g.nx;
  gr->nblk = (int)((L + roi_block_pixels() - 1) / roi_block_pixels());
  gr->Kpad = (int)(((L + 31) / 32) * 32);
  const size_t nb = (size_t)g.G * g.ns * b;
  if ((s = m.alloc(&gr->blockcount, gr->nblk)) || (s = m.alloc(&gr->blockoff, gr->nblk)) ||
      (s = m.alloc(&gr->dK, 1)) || (s = m.alloc(&gr->pix, L)) || (s = m.alloc(&gr->chat, (size_t)g.nc * gr->Kpad)) ||
      (s = m.alloc(&gr->dT, (size_t)g.nc * g.nc)) || (s = m.alloc(&gr->d_ref, g.G)) ||
      (s = m.alloc(&gr->P, (size_t)g.G * g.ns * g.ns)) || (s = m.alloc(&gr->X, nb)) || (s = m.alloc(&gr->Y, nb)) ||
      (s = m.alloc(&gr->U, nb)) || (s = m.alloc(&gr->Hm, (size_t)g.G * b * b)) ||
      (s = m.alloc(&gr->W, (size_t)g.G * b * b)) || (s = m.alloc(&gr->ritz, (size_t)g.G * b)) ||
      (s = m.alloc(&gr->order, (size_t)g.G * b)) || (s = m.alloc(&gr->resid, (size_t)g.G)) ||
      (s = m.alloc(&gr->P32, (size_t)g.G * g.ns * g.ns)) || (s = m.alloc(&gr->X32, nb)) ||
      (s = m.alloc(&gr->Y32, nb)))
    return s;
  CK(cudaMemcpy(gr->d_ref, plan->ref.data(), sizeof(int) * g.G, cudaMemcpyHostToDevice));
  {
    const char* e = getenv("GPJC_SIMT_GRAM");
    gr->tc_gram = !(e && e[0] == '1') && tc_gram2_smem(g) <= 227 * 1024;
    std::vector<int2> pairs;
    for (int n = 0; n < g.nc; ++n)
      for (int n2 = n; n2 < g.nc; ++n2) pairs.push_back(make_int2(n, n2));
    gr->tg_npairs = (int)pairs.size();
    if ((s = m.upload(&gr->tg_pairs, pairs))) return s;
    if (!gr->tc_status) {
      if ((s = m.alloc(&gr->tc_status, 1))) return s;
      CK(cudaMemset(gr->tc_status, 0, sizeof(int)));
    }
  }
  if ((s = groups_compute(gr, (const float2*)d_coil, d_roi, h_T, st))) return s;
  // the ROI must not be empty: checked once here (later rebuilds are asynchronous)
  CK(cudaStreamSynchronize(st));
  if ((s = groups_sync_host(gr))) return s;
  if (gr->K <= 0) return fail(GPJC_EINVAL, "ROI is empty (or no coil sees it)");
  *out = guard.release();
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_groups_rebuild(gpjc_groups* gr, const float* d_coil, const uint8_t* d_roi,
                                           const float* h_T, void* stream) {
  if (!gr || !d_coil || !d_roi) return fail(GPJC_EINVAL, "null argument");
  if (!gr->built) return fail(GPJC_EINVAL, "groups were created from matrices");
  return groups_compute(gr, (const float2*)d_coil, d_roi, h_T, (cudaStream_t)stream);
}

extern "C" gpjc_status gpjc_groups_from_matrices(const gpjc_plan* plan, const float* h_A, gpjc_groups** out) {
  if (!plan || !h_A || !out) return fail(GPJC_EINVAL, "null argument");
  *out = nullptr;
  auto* gr = new (std::nothrow) gpjc_groups();
  if (!gr) return fail(GPJC_ENOMEM, "host allocation");
  std::unique_ptr<gpjc_groups> guard(gr);
  gr->plan = plan;
  gr->b = 0;
  gr->K = 0;
  gr->max_resid = 0.0;
  gr->built = false;
  gr->host_valid = true;
  gr->P = nullptr;
  gr->pix = nullptr;
  gpjc_status s;
  if ((s = groups_alloc_A(gr))) return s;
  const size_t na = (size_t)plan->aoff.back() + (size_t)plan->ns * plan->keep.back();
  std::vector<float2> hA(na), hAT(na);
  memcpy(hA.data(), h_A, sizeof(float2) * na);
  std::vector<float> sc(plan->G, 0.f);
  for (int g = 0; g < plan->G; ++g) {
    const int kg = plan->keep[g];
    for (int k = 0; k < kg; ++k)
      for (int i = 0; i < plan->ns; ++i) {
        const float2 v = hA[plan->aoff[g] + (size_t)k * plan->ns + i];
        if (!std::isfinite(v.x) || !std::isfinite(v.y)) return fail(GPJC_EINVAL, "non-finite A entry (group %d)", g);
        hAT[plan->aoff[g] + (size_t)i * kg + k] = v;
        sc[g] = std::max(sc[g], std::max(std::fabs(v.x), std::fabs(v.y)));
      }
  }
  CK(cudaMemcpy(gr->A, hA.data(), sizeof(float2) * na, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(gr->AT, hAT.data(), sizeof(float2) * na, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(gr->scale, sc.data(), sizeof(float) * sc.size(), cudaMemcpyHostToDevice));
  if ((s = groups_pack_tc(gr, 0))) return s;
  CK(cudaDeviceSynchronize());
  *out = guard.release();
  return GPJC_OK;
}

extern "C" void gpjc_groups_destroy(gpjc_groups* groups) { delete groups; }

extern "C" gpjc_status gpjc_groups_info_get(const gpjc_groups* gr, gpjc_groups_info* info) {
  if (!gr || !info) return fail(GPJC_EINVAL, "null argument");
  gpjc_status s = groups_sync_host(gr);
  if (s) return s;
  info->roi_pixels = gr->K;
  info->block = gr->b;
  info->max_residual = gr->max_resid;
  return GPJC_OK;
}

// Gradient of the smoothed TV of Eq. 17 (Sec. 3.4: TV by a smooth
// approximation), per z-slice.  Asynchronous on `stream`.
extern "C" gpjc_status gpjc_tv_grad(const float* d_x, int32_t nz, int32_t ny, int32_t nx, double eps, float* d_g,
                                    void* stream) {
  if (!d_x || !d_g) return fail(GPJC_EINVAL, "null argument");
  if (nz < 1 || ny < 1 || nx < 1) return fail(GPJC_EINVAL, "image dimensions must be >= 1");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(GPJC_EINVAL, "eps must be finite and > 0");
  // the kernel works with eps^2 in FP32: it must be a normal positive float
  // (a zero or subnormal eps^2 makes flat regions divide by zero)
  const double eps2 = eps * eps;
  if (!(eps2 >= (double)FLT_MIN) || !(eps2 <= (double)FLT_MAX))
    return fail(GPJC_EINVAL, "eps^2 = %g is not a normal FP32 number", eps2);
  if ((const void*)d_x == (const void*)d_g) return fail(GPJC_EINVAL, "d_g must not alias d_x");
  CK(launch_tv_grad((const float2*)d_x, (float2*)d_g, nz, ny, nx, (float)eps2, (cudaStream_t)stream));
  return GPJC_OK;
}

// Kept dimension per group from the leading eigenvalues (Eq. 8; Sec. 2.4:
// the spectrum of P_g indicates N_s'): the smallest k whose leading values
// hold `threshold` of trace(P_g).  Host only.
extern "C" gpjc_status gpjc_keep_from_energy(const double* h_eig, int32_t n_groups, int32_t m, const double* h_trace,
                                             double threshold, int32_t* h_keep) {
  if (!h_eig || !h_keep) return fail(GPJC_EINVAL, "null argument");
  if (n_groups < 1 || m < 1) return fail(GPJC_EINVAL, "n_groups and m must be >= 1");
  if (!(threshold > 0.0 && threshold <= 1.0)) return fail(GPJC_EINVAL, "threshold must be in (0, 1]");
  for (int64_t i = 0; i < (int64_t)n_groups * m; ++i)
    if (!std::isfinite(h_eig[i])) return fail(GPJC_ENONFINITE, "non-finite eigenvalue at %lld", (long long)i);
  if (h_trace)
    for (int g = 0; g < n_groups; ++g)
      if (!std::isfinite(h_trace[g]) || h_trace[g] < 0.0) return fail(GPJC_EINVAL, "trace of group %d", g);
  for (int g = 0; g < n_groups; ++g) {
    const double* ev = h_eig + (size_t)g * m;
    double tr = 0.0;
    if (h_trace) {
      tr = h_trace[g];
    } else {
      for (int k = 0; k < m; ++k) tr += std::max(ev[k], 0.0);  // index order
    }
    const double target = threshold * tr;
    double acc = 0.0;
    h_keep[g] = -1;
    for (int k = 0; k < m; ++k) {
      acc += std::max(ev[k], 0.0);
      if (acc >= target) {
        h_keep[g] = k + 1;
        break;
      }
    }
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_groups_get(const gpjc_groups* gr, float* h_A, double* h_ritz) {
  if (!gr) return fail(GPJC_EINVAL, "null groups");
  const gpjc_plan* p = gr->plan;
  const size_t na = (size_t)p->aoff.back() + (size_t)p->ns * p->keep.back();
  gpjc_status s = groups_sync_host(gr);
  if (s) return s;
  if (h_A) CK(cudaMemcpy(h_A, gr->A, sizeof(float2) * na, cudaMemcpyDeviceToHost));
  if (h_ritz && !gr->ritz_h.empty()) std::copy(gr->ritz_h.begin(), gr->ritz_h.end(), h_ritz);
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_groups_gram(const gpjc_groups* gr, double* h_P) {
  if (!gr || !h_P) return fail(GPJC_EINVAL, "null argument");
  if (!gr->P || !gr->keep_gram) return fail(GPJC_EINVAL, "groups were built without keep_gram");
  const gpjc_plan* p = gr->plan;
  CK(cudaMemcpy(h_P, gr->P, sizeof(double2) * (size_t)p->G * p->ns * p->ns, cudaMemcpyDeviceToHost));
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_groups_roi(const gpjc_groups* gr, int32_t* h_pix) {
  if (!gr || !h_pix) return fail(GPJC_EINVAL, "null argument");
  gpjc_status s = groups_sync_host(gr);
  if (s) return s;
  if (gr->K <= 0) return fail(GPJC_EINVAL, "groups were not built from a ROI");
  CK(cudaMemcpy(h_pix, gr->pix, sizeof(int) * (size_t)gr->K, cudaMemcpyDeviceToHost));
  return GPJC_OK;
}

// ------------------------------------------------------------------ compress --
extern "C" gpjc_status gpjc_compress(const gpjc_groups* gr, const float* d_S, float* d_Sc, gpjc_precision prec,
                                     void* stream) {
  if (!gr || !d_S || !d_Sc) return fail(GPJC_EINVAL, "null argument");
  const Geo& g = gr->plan->geo;
  if (prec == GPJC_FP32) {
    CK(launch_compress_fp32(g, (const float2*)d_S, g.n_lines, gr->AT, (float2*)d_Sc, (cudaStream_t)stream));
    return GPJC_OK;
  }
  if (prec != GPJC_BF16 && prec != GPJC_FP16) return fail(GPJC_EINVAL, "unknown precision");
  const gpjc_plan* p = gr->plan;
  if (!p->tc_ok) return fail(GPJC_EUNSUPPORTED, "tensor-core compression needs a periodic group map");
  if (((uintptr_t)d_S) & 15) return fail(GPJC_EINVAL, "d_S must be 16-byte aligned");
  TcGeom t = prec == GPJC_BF16 ? p->tc32b : p->tc32h;
  t.scale = gr->scale;
  CUtensorMap map;
  if (!make_tc_tmap(t, d_S, g.n_lines, 4, &map)) return fail(GPJC_ECUDA, "cuTensorMapEncodeTiled failed");
  const int fmt = prec == GPJC_BF16 ? 1 : 0;
  CK(launch_tc_compress(map, t, fmt, 4, gr->tc_bc[fmt], (float2*)d_Sc, 0, g.n_lines, gr->tc_status,
                        (cudaStream_t)stream));
  return GPJC_OK;
}

// ------------------------------------------------------------------ operator --
enum { SC_BB = 0, SC_QQ = 1, SC_RR0 = 2, SC_RR1 = 3, SC_NV = 4, SC_LIP = 5, SC_TMP = 6, SC_N = 16 };

struct gpjc_op {
  const gpjc_groups* gr;
  const gpjc_plan* plan;
  const float2* coil;
  gpjc_precision prec;
  int nchunk, nchunk_max;      // coil chunks of the forward readout (partial Hpart planes)
  int nchunk_a, nchunk_a_max;  // coil chunks of the adjoint readout (partial images in xparts)
  int adj_pieces;             // 16-bit operators: row pieces of the adjoint readout (V stays in L2)
  size_t L;
  float2 *Hpart, *T, *H2, *xparts;
  float2 *vb, *vr, *vp, *vy, *vv, *vtmp;
  float2 *V, *TV;  // lazily allocated (simulation)
  void* V16;       // 16-bit hybrid data [rows][nc][ntx] of the tensor-core operator
  bool tc_ro;      // readout stage on the tensor cores (16-bit operators, w >= 8; see tc_readout)
  CUtensorMap map16;
  double* partials;
  int npartials;
  unsigned* counter;
  double* sc;
  double* hist;
  int hist_len;
  double* ds_rowval;  // per-set CG: one FP64 sum per image row
  double* ds_sc;      // per-set CG: ||r||^2 (two, ping-pong) and <p, N p> per aliased set
  int* status;
  DevMem mem;
  DevMem lazy;
  // cached recon graph; captured and replayed on a private stream that is
  // ordered after / before the caller's stream with events (the legacy
  // default stream cannot be captured)
  cudaGraphExec_t gexec;
  std::vector<char> gkey;
  int graph_kernels;
  cudaStream_t cap_st;
  cudaEvent_t ev_in, ev_out;
  bool legacy_readout;  // use the per-output readout kernels (set by GPJC_LEGACY_READOUT=1)
  // nonlinear local-B0 operator: stored compressed readout matrices
  // [rows][ntx_c][nx] replace the FFT readout stage (nullptr: wave operator)
  float2* lb0_G;
  // optional per-stage timing with events (GPJC_STAGE_*)
  bool prof_on;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used;
  std::vector<std::pair<int, size_t>> prof_marks;  // (stage, index of start event)
};

// records the start / end of a stage when profiling is on
static void prof_begin(gpjc_op* op, int stage, cudaStream_t st, size_t* mark) {
  *mark = (size_t)-1;
  if (!op->prof_on || op->prof_used + 2 > op->prof_pool.size()) return;
  *mark = op->prof_used;
  op->prof_used += 2;
  op->prof_marks.push_back({stage, *mark});
  // inside a capture the record must become an event node of the graph
  cudaEventRecordWithFlags(op->prof_pool[*mark], st, g_capturing ? cudaEventRecordExternal : 0);
}
static void prof_end(gpjc_op* op, cudaStream_t st, size_t mark) {
  if (mark != (size_t)-1)
    cudaEventRecordWithFlags(op->prof_pool[mark + 1], st, g_capturing ? cudaEventRecordExternal : 0);
}

// adjoint readout: enough (row block, coil chunk) blocks for three
// resident blocks on each of the 152 SMs
static int auto_nchunk_adj(const gpjc_plan* p) {
  const int rows = p->ny * p->nz;
  const int rb = p->rt_a.rb ? p->rt_a.rb : 1;
  const int blocks = (rows + rb - 1) / rb;
  int n = 1;
  while (blocks * n < 3 * 152 && n * 2 <= p->nc) n *= 2;
  return n;
}

// 16-bit operators: the adjoint expands A_g^H H into FP32 spectra
// [rows][nc][ntx] before the inverse readout FFT; in row pieces of at most
// ~40 MB of spectra each, the spectra are read back from L2 instead of HBM
constexpr int kMaxAdjPieces = 8;
static int auto_adj_pieces(const gpjc_plan* p) {
  const double bytes = 8.0 * p->ny * p->nz * p->nc * p->os * p->nx;
  int n = 1;
  while (bytes / n > 40e6 && n < kMaxAdjPieces) n *= 2;
  return n;
}

static int auto_nchunk(const gpjc_plan* p) {
  const int rows = p->ny * p->nz;
  int n = 1;
  while ((long long)rows * n < 1024 && n * 2 <= p->nc) n *= 2;
  return n;
}

// Whether a 16-bit operator runs its readout stage on the tensor cores
// (k1_sim_* spectra + k_tc_compress / k_tc_expand) or on the FP32
// register-tiled kernels of the FP32 operator.  Patches narrower than 8
// samples give the compression GEMM TMA boxes of 16-32 bytes and a K of
// nc w per group: on the 224 x 224 x 160 volume with per-period groups of
// w = 2 the tensor-core readout ran at 0.56x the FP32 one (compression and
// expansion kernels ~10x off their HBM traffic) while saving a contraction
// of two taps per patch, and its spectra buffer took 12 GB.
// GPJC_TC_READOUT=0 / 1 forces either.
static bool tc_readout(const gpjc_plan* p, gpjc_precision prec) {
  if (prec == GPJC_FP32) return false;
  if (const char* e = getenv("GPJC_TC_READOUT")) {
    if (e[0] == '0') return false;
    if (e[0] == '1') return true;
  }
  return p->w >= 8;
}

// Workspace layout of an operator: chunk counts and element counts of every
// device buffer gpjc_op_create allocates (shared with gpjc_query).
struct OpSizes {
  int nchunk, nchunk_max, nchunk_a, nchunk_a_max, adj_pieces;
  size_t L, HN, npartials, hist_len, spectra;
  size_t bytes;  // total device bytes
};
static OpSizes op_sizes(const gpjc_plan* p, gpjc_precision prec, int nchunk) {
  OpSizes z{};
  const Geo& g = p->geo;
  z.nchunk = nchunk > 0 ? nchunk : auto_nchunk(p);
  // workspaces sized for the largest chunk count the autotuner may pick
  int nmax = z.nchunk;
  {
    int n = 1;
    while (n * 2 <= p->nc && n * 2 <= 16) n *= 2;
    const size_t per = (size_t)p->ny * p->nz * std::max(p->ntxc, p->nx) * sizeof(float2);
    while (n > nmax && (size_t)n * per > ((size_t)4 << 30)) n /= 2;
    nmax = std::max(nmax, n);
  }
  z.nchunk_max = nmax;
  z.L = (size_t)g.rows * g.nx;
  // the adjoint's partial images are small: allow up to nc chunks (1 GB cap)
  {
    int n = 1;
    while (n * 2 <= p->nc && (size_t)n * 2 * z.L * sizeof(float2) <= ((size_t)1 << 30)) n *= 2;
    z.nchunk_a_max = std::max(n, nmax);
    z.nchunk_a = std::min(auto_nchunk_adj(p), z.nchunk_a_max);
    z.adj_pieces = auto_adj_pieces(p);
    // GPJC_ADJ_PIECES=n (1..8) overrides the default split (the results do
    // not depend on it: whole expansion row tiles per piece)
    if (const char* e = getenv("GPJC_ADJ_PIECES")) {
      const int v = atoi(e);
      if (v >= 1 && v <= kMaxAdjPieces) z.adj_pieces = v;
    }
  }
  z.HN = (size_t)g.rows * g.ntxc;
  z.npartials = std::max(pe_normal_blocks(g, g.ntxc), sum_parts_blocks(z.L)) + 16;
  z.hist_len = (size_t)1 << 14;
  z.spectra = tc_readout(p, prec) ? (size_t)g.rows * g.nc * g.ntx : 0;
  const size_t c64 = z.HN * nmax + z.HN + z.L * (size_t)z.nchunk_a_max + 6 * z.L + (g.dim3d ? z.HN : 0) + z.spectra;
  z.bytes = sizeof(float2) * c64 + sizeof(double) * (z.npartials + SC_N + z.hist_len) + 4 * sizeof(unsigned) +
            4 * sizeof(int) + sizeof(double) * ((size_t)g.rows + 3 * (size_t)p->n_sets);
  return z;
}

extern "C" gpjc_status gpjc_probe_fp32_tflops(int32_t iters, double* tflops) {
  if (!tflops || iters < 1) return fail(GPJC_EINVAL, "tflops must be non-NULL and iters >= 1");
  CK(probe_fma_tflops(iters, tflops));
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_query(const gpjc_groups* gr, gpjc_precision prec, int32_t nchunk, int32_t* ntx_c,
                                  uint64_t* workspace_bytes) {
  if (!gr) return fail(GPJC_EINVAL, "null groups");
  if (prec != GPJC_FP32 && prec != GPJC_BF16 && prec != GPJC_FP16) return fail(GPJC_EINVAL, "unknown precision");
  const gpjc_plan* p = gr->plan;
  if (nchunk < 0 || nchunk > p->nc) return fail(GPJC_EINVAL, "nchunk must be in [0, nc]");
  if (prec != GPJC_FP32 && !p->tc_ok)
    return fail(GPJC_EUNSUPPORTED, "the tensor-core operator needs a periodic group map");
  if (ntx_c) *ntx_c = p->ntxc;
  if (workspace_bytes) *workspace_bytes = (uint64_t)op_sizes(p, prec, nchunk).bytes;
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_op_create(const gpjc_groups* gr, const float* d_coil, gpjc_precision prec,
                                      int32_t nchunk, gpjc_op** out) {
  if (!gr || !d_coil || !out) return fail(GPJC_EINVAL, "null argument");
  *out = nullptr;
  if (prec != GPJC_FP32 && prec != GPJC_BF16 && prec != GPJC_FP16) return fail(GPJC_EINVAL, "unknown precision");
  const gpjc_plan* p = gr->plan;
  if (prec != GPJC_FP32 && !p->tc_ok)
    return fail(GPJC_EUNSUPPORTED, "the tensor-core operator needs a periodic group map");
  if (nchunk < 0 || nchunk > p->nc) return fail(GPJC_EINVAL, "nchunk must be in [0, nc]");
  auto* op = new (std::nothrow) gpjc_op();
  if (!op) return fail(GPJC_ENOMEM, "host allocation");
  std::unique_ptr<gpjc_op> guard(op);
  op->gr = gr;
  op->plan = p;
  op->coil = (const float2*)d_coil;
  op->prec = prec;
  op->tc_ro = tc_readout(p, prec);
  const OpSizes z = op_sizes(p, prec, nchunk);
  op->nchunk = z.nchunk;
  const int nmax = z.nchunk_max;
  op->nchunk_max = nmax;
  const Geo& g = p->geo;
  op->L = z.L;
  op->nchunk_a_max = z.nchunk_a_max;
  op->nchunk_a = z.nchunk_a;
  op->adj_pieces = z.adj_pieces;
  const size_t HN = z.HN;
  gpjc_status s;
  DevMem& m = op->mem;
  if ((s = m.alloc(&op->Hpart, HN * nmax)) || (s = m.alloc(&op->H2, HN)) ||
      (s = m.alloc(&op->xparts, op->L * (size_t)op->nchunk_a_max)) || (s = m.alloc(&op->vb, op->L)) ||
      (s = m.alloc(&op->vr, op->L)) || (s = m.alloc(&op->vp, op->L)) || (s = m.alloc(&op->vy, op->L)) ||
      (s = m.alloc(&op->vv, op->L)) || (s = m.alloc(&op->vtmp, op->L)))
    return s;
  op->T = nullptr;
  if (g.dim3d && (s = m.alloc(&op->T, HN))) return s;
  op->npartials = (int)z.npartials;
  op->hist_len = (int)z.hist_len;
  if ((s = m.alloc(&op->ds_rowval, (size_t)g.rows)) || (s = m.alloc(&op->ds_sc, 3 * (size_t)p->n_sets)))
    return s;
  if ((s = m.alloc(&op->partials, op->npartials)) || (s = m.alloc(&op->counter, 4)) ||
      (s = m.alloc(&op->sc, SC_N)) || (s = m.alloc(&op->hist, op->hist_len)) || (s = m.alloc(&op->status, 4)))
    return s;
  CK(cudaMemset(op->counter, 0, 4 * sizeof(unsigned)));
  CK(cudaMemset(op->sc, 0, SC_N * sizeof(double)));
  CK(cudaMemset(op->status, 0, 4 * sizeof(int)));
  op->V = op->TV = nullptr;
  op->V16 = nullptr;
  if (op->tc_ro) {
    // one buffer serves the forward spectra (FP16, or FP32 for the split BF16
    // compression) and the FP32 adjoint spectra
    float2* v16;
    if ((s = m.alloc(&v16, z.spectra))) return s;
    op->V16 = v16;
    const bool f32src = prec == GPJC_BF16;
    if (!make_tc_tmap(f32src ? p->tc32b : p->tc16, op->V16, g.rows, f32src ? 4 : 2, &op->map16))
      return fail(GPJC_ECUDA, "cuTensorMapEncodeTiled failed");
  }
  op->gexec = nullptr;
  op->graph_kernels = 0;
  op->lb0_G = nullptr;
  {
    const char* e = getenv("GPJC_LEGACY_READOUT");
    op->legacy_readout = e && e[0] == '1';
  }
  op->prof_on = false;
  op->prof_used = 0;
  op->cap_st = nullptr;
  op->ev_in = op->ev_out = nullptr;
  CK(cudaStreamCreateWithFlags(&op->cap_st, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&op->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&op->ev_out, cudaEventDisableTiming));
  *out = guard.release();
  return GPJC_OK;
}

// Nonlinear local-B0 operator (Sec. 2.1-2.2, Eq. 2-3, 14): an FP32 operator
// whose readout stage applies stored compressed readout matrices built here
// from A_g, the coil maps and the local-B0 phase sum_l a_l(t) B_l(r).
extern "C" gpjc_status gpjc_op_create_local_b0(const gpjc_groups* gr, const float* d_coil, int32_t n_fields,
                                               const float* d_fields, const double* h_amps, gpjc_op** out) {
  if (!gr || !d_coil || !out || (n_fields > 0 && (!d_fields || !h_amps)))
    return fail(GPJC_EINVAL, "null argument");
  *out = nullptr;
  if (n_fields < 0 || n_fields > 64) return fail(GPJC_EINVAL, "n_fields must be in [0, 64]");
  const gpjc_plan* p = gr->plan;
  const Geo& g = p->geo;
  if (lb0_build_tile(g.ns) < 1) return fail(GPJC_EUNSUPPORTED, "N_s too large for the matrix build");
  for (size_t i = 0; i < (size_t)n_fields * g.ntx; ++i)
    if (!std::isfinite(h_amps[i])) return fail(GPJC_EINVAL, "amplitudes must be finite");
  gpjc_op* op = nullptr;
  gpjc_status s = gpjc_op_create(gr, d_coil, GPJC_FP32, 1, &op);
  if (s) return s;
  std::unique_ptr<gpjc_op, void (*)(gpjc_op*)> guard(op, gpjc_op_destroy);
  op->nchunk = 1;
  // adjoint: enough (column chunk, row) blocks for two per SM, at least 32
  // columns per chunk
  {
    int n = 1;
    while (g.rows * n < 2 * 152 && n * 2 <= op->nchunk_a_max && g.ntxc / (n * 2) >= 32) n *= 2;
    op->nchunk_a = n;
  }
  std::vector<float> amps((size_t)std::max(n_fields, 1) * g.ntx, 0.f);
  for (size_t i = 0; i < (size_t)n_fields * g.ntx; ++i) amps[i] = (float)h_amps[i];
  float* d_amps = nullptr;
  float2* G = nullptr;
  if ((s = op->mem.upload(&d_amps, amps)) || (s = op->mem.alloc(&G, (size_t)g.rows * g.ntxc * g.nx))) return s;
  CK(launch_lb0_build(g, n_fields, (const float2*)d_coil, d_fields, d_amps, gr->A, G, 0));
  CK(cudaDeviceSynchronize());
  op->lb0_G = G;
  *out = guard.release();
  return GPJC_OK;
}

extern "C" void gpjc_op_destroy(gpjc_op* op) {
  if (!op) return;
  if (op->gexec) cudaGraphExecDestroy(op->gexec);
  if (op->cap_st) {
    cudaStreamSynchronize(op->cap_st);
    cudaStreamDestroy(op->cap_st);
  }
  if (op->ev_in) cudaEventDestroy(op->ev_in);
  if (op->ev_out) cudaEventDestroy(op->ev_out);
  for (cudaEvent_t e : op->prof_pool) cudaEventDestroy(e);
  delete op;
}

// The forward readout runs the balanced k1f_batched launch (partial sums in
// bal_planes planes instead of one per coil chunk; the forward chunk knob
// then has no effect).
static bool fwd_balanced(const gpjc_op* op) {
  const RTiles& rt = op->plan->rt_f;
  return !op->lb0_G && !op->tc_ro && !op->legacy_readout && rt.rb && rt.nb && rt.bal_units > 0 &&
         rt.bal_planes <= op->nchunk_max;
}
// partial planes of Hpart the phase-encode stage sums after the forward readout
static int fwd_planes(const gpjc_op* op) {
  if (op->tc_ro) return 1;
  return fwd_balanced(op) ? op->plan->rt_f.bal_planes : op->nchunk;
}

// --- internal launch sequences (no validation) ---
// readout stage of E_c into op->Hpart (register-tiled kernel when the plan has
// tiles; 16-bit hybrid data + tensor-core compression for BF16 / FP16
// operators whose readout runs on the tensor cores)
static cudaError_t readout_fwd(const gpjc_op* op, const float2* x, cudaStream_t st) {
  const gpjc_plan* p = op->plan;
  if (op->lb0_G) return launch_lb0_fwd(p->geo, op->lb0_G, x, op->Hpart, st);
  if (op->tc_ro) {
    // BF16: FP32 spectra, split into head + remainder by the compression GEMM;
    // FP16: FP16 spectra, one rounding
    const int fmt = op->prec == GPJC_BF16 ? 1 : 0;
    TcGeom t = fmt ? p->tc32b : p->tc16;
    t.scale = op->gr->scale;
    // one piece of all rows: smaller pieces keep their spectra in L2 but
    // launch fewer blocks each, which cost more on the 256 x 256 workload
    // (1 / 2 / 4 pieces: 158 / 171 / 240 us per BF16 application)
    const Geo& g = p->geo;
    const int per = g.rows;
    for (int r0 = 0; r0 < g.rows; r0 += per) {
      const int nr = std::min(per, g.rows - r0);
      cudaError_t e = fmt ? launch_sim_fwd_rows(g, x, op->coil, (float2*)op->V16, op->nchunk, r0, nr, st)
                          : launch_sim_fwd_f16(g, x, op->coil, op->V16, op->nchunk, r0, nr, st);
      if (e != cudaSuccess) return e;
      e = launch_tc_compress(op->map16, t, fmt, fmt ? 4 : 2, op->gr->tc_bc[fmt], op->Hpart, r0, r0 + nr, op->status,
                             st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (p->rt_f.rb && !op->legacy_readout) {
    if (p->rt_f.nb)
      return launch_k1f_batched(p->geo, p->rt_f, x, op->coil, op->gr->AT, op->Hpart, op->nchunk, fwd_balanced(op),
                                st);
    return launch_k1f_tiled(p->geo, p->rt_f, x, op->coil, op->gr->AT, op->Hpart, op->nchunk, st);
  }
  return launch_k1_fwd_fp32(p->geo, x, op->coil, op->gr->AT, op->Hpart, op->nchunk, st);
}
// readout stage of E_c^H from op->H2 into op->xparts
static cudaError_t readout_adj(const gpjc_op* op, cudaStream_t st) {
  const gpjc_plan* p = op->plan;
  if (op->lb0_G) return launch_lb0_adj(p->geo, op->lb0_G, op->H2, op->xparts, op->nchunk_a, st);
  if (op->tc_ro) {
    const int fmt = op->prec == GPJC_BF16 ? 1 : 0;
    TcGeom t = p->tc16;
    t.scale = op->gr->scale;
    const Geo& g = p->geo;
    // pieces of whole expansion row tiles
    const int tiles = (g.rows + t.lt - 1) / t.lt;
    const int per = (tiles + op->adj_pieces - 1) / op->adj_pieces * t.lt;
    for (int r0 = 0; r0 < g.rows; r0 += per) {
      const int nr = std::min(per, g.rows - r0);
      cudaError_t e = launch_tc_expand(t, fmt, op->H2 + (size_t)r0 * g.ntxc, op->gr->tc_bx[fmt],
                                       (float2*)op->V16 + (size_t)r0 * g.nc * g.ntx, nr, op->status, st);
      if (e != cudaSuccess) return e;
      e = launch_sim_adj_rows(g, (const float2*)op->V16, op->coil, op->xparts, op->nchunk_a, r0, nr, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (p->rt_a.rb && !op->legacy_readout)
    return launch_k1a_tiled(p->geo, p->rt_a, op->H2, op->coil, op->gr->A, op->xparts, op->nchunk_a, st);
  return launch_k1_adj_fp32(p->geo, op->H2, op->coil, op->gr->A, op->xparts, op->nchunk_a, st);
}

static gpjc_status op_fwd(const gpjc_op* cop, const float2* x, float2* y, cudaStream_t st) {
  gpjc_op* op = const_cast<gpjc_op*>(cop);
  const Geo& g = op->plan->geo;
  size_t m;
  prof_begin(op, GPJC_STAGE_READOUT_FWD, st, &m);
  CK(readout_fwd(op, x, st));
  prof_end(op, st, m);
  prof_begin(op, GPJC_STAGE_PHASE_ENCODE, st, &m);
  CK(launch_pe_fwd(g, op->Hpart, fwd_planes(op), g.ntxc, op->T, y, st));
  prof_end(op, st, m);
  return GPJC_OK;
}

static gpjc_status op_adj_parts(const gpjc_op* cop, const float2* y, cudaStream_t st) {
  gpjc_op* op = const_cast<gpjc_op*>(cop);
  const Geo& g = op->plan->geo;
  size_t m;
  prof_begin(op, GPJC_STAGE_PHASE_ENCODE, st, &m);
  CK(launch_pe_adj(g, y, g.ntxc, op->T, op->H2, st));
  prof_end(op, st, m);
  prof_begin(op, GPJC_STAGE_READOUT_ADJ, st, &m);
  CK(readout_adj(op, st));
  prof_end(op, st, m);
  return GPJC_OK;
}

// xparts <- chunks of E_c^H E_c x ; *qq <- ||E_c x||^2 (if qq)
static gpjc_status op_normal_parts(const gpjc_op* cop, const float2* x, double* qq, cudaStream_t st) {
  gpjc_op* op = const_cast<gpjc_op*>(cop);
  const Geo& g = op->plan->geo;
  size_t m;
  prof_begin(op, GPJC_STAGE_READOUT_FWD, st, &m);
  CK(readout_fwd(op, x, st));
  prof_end(op, st, m);
  prof_begin(op, GPJC_STAGE_PHASE_ENCODE, st, &m);
  CK(launch_pe_normal(g, op->Hpart, fwd_planes(op), g.ntxc, op->T, op->H2, op->partials,
                      op->counter, qq, st));
  prof_end(op, st, m);
  prof_begin(op, GPJC_STAGE_READOUT_ADJ, st, &m);
  CK(readout_adj(op, st));
  prof_end(op, st, m);
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_apply_E(const gpjc_op* op, const float* d_x, float* d_y, void* stream) {
  if (!op || !d_x || !d_y) return fail(GPJC_EINVAL, "null argument");
  return op_fwd(op, (const float2*)d_x, (float2*)d_y, (cudaStream_t)stream);
}

extern "C" gpjc_status gpjc_apply_EH(const gpjc_op* op, const float* d_y, float* d_x, void* stream) {
  if (!op || !d_x || !d_y) return fail(GPJC_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  gpjc_status s = op_adj_parts(op, (const float2*)d_y, st);
  if (s) return s;
  CK(launch_sum_parts(op->xparts, op->nchunk_a, op->L, (float2*)d_x, nullptr, nullptr, nullptr, st));
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_apply_normal(const gpjc_op* op, const float* d_x, float* d_out, double* d_qq,
                                         void* stream) {
  if (!op || !d_x || !d_out) return fail(GPJC_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  gpjc_status s = op_normal_parts(op, (const float2*)d_x, d_qq, st);
  if (s) return s;
  CK(launch_sum_parts(op->xparts, op->nchunk_a, op->L, (float2*)d_out, nullptr, nullptr, nullptr, st));
  return GPJC_OK;
}

static gpjc_status ensure_sim_buffers(gpjc_op* op) {
  const Geo& g = op->plan->geo;
  const size_t n = (size_t)g.rows * g.nc * g.ntx;
  gpjc_status s;
  if (!op->V && (s = op->lazy.alloc(&op->V, n))) return s;
  if (g.dim3d && !op->TV && (s = op->lazy.alloc(&op->TV, n))) return s;
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_simulate(const gpjc_op* cop, const float* d_x, float* d_S, void* stream) {
  if (!cop || !d_x || !d_S) return fail(GPJC_EINVAL, "null argument");
  if (cop->lb0_G) return fail(GPJC_EUNSUPPORTED, "the uncompressed model is the wave model's (local-B0 operator)");
  gpjc_op* op = const_cast<gpjc_op*>(cop);
  gpjc_status s = ensure_sim_buffers(op);
  if (s) return s;
  const Geo& g = op->plan->geo;
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_sim_fwd(g, (const float2*)d_x, op->coil, op->V, op->nchunk, st));
  CK(launch_pe_fwd(g, op->V, 1, g.nc * g.ntx, op->TV, (float2*)d_S, st));
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_simulate_adjoint(const gpjc_op* cop, const float* d_S, float* d_x, void* stream) {
  if (!cop || !d_x || !d_S) return fail(GPJC_EINVAL, "null argument");
  if (cop->lb0_G) return fail(GPJC_EUNSUPPORTED, "the uncompressed model is the wave model's (local-B0 operator)");
  gpjc_op* op = const_cast<gpjc_op*>(cop);
  gpjc_status s = ensure_sim_buffers(op);
  if (s) return s;
  const Geo& g = op->plan->geo;
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_pe_adj(g, (const float2*)d_S, g.nc * g.ntx, op->TV, op->V, st));
  CK(launch_sim_adj(g, op->V, op->coil, op->xparts, op->nchunk_a, st));
  CK(launch_sum_parts(op->xparts, op->nchunk_a, op->L, (float2*)d_x, nullptr, nullptr, nullptr, st));
  return GPJC_OK;
}

// times one application of E_c^H E_c (both readout stages, the phase-encode
// stage and the sum of the partial images) with the current chunk counts
// (best of three runs of five applications, after one warm-up application)
static gpjc_status time_normal(gpjc_op* op, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  gpjc_status s;
  *ms = 1e30f;
  for (int trial = 0; trial < 4; ++trial) {
    if (trial > 0) CK(cudaEventRecord(e0, st));
    for (int r = 0; r < (trial > 0 ? 5 : 1); ++r) {
      if ((s = op_normal_parts(op, op->vv, nullptr, st))) return s;
      CK(launch_sum_parts(op->xparts, op->nchunk_a, op->L, op->vtmp, nullptr, nullptr, nullptr, st));
    }
    if (trial == 0) continue;
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    *ms = std::min(*ms, t);
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_op_tuning(const gpjc_op* op, int32_t* nchunk, int32_t* nchunk_adj, int32_t* adj_pieces) {
  if (!op) return fail(GPJC_EINVAL, "null operator");
  if (nchunk) *nchunk = op->nchunk;
  if (nchunk_adj) *nchunk_adj = op->nchunk_a;
  if (adj_pieces) *adj_pieces = op->adj_pieces;
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_op_set_tuning(gpjc_op* op, int32_t nchunk, int32_t nchunk_adj, int32_t adj_pieces) {
  if (!op) return fail(GPJC_EINVAL, "null operator");
  if (op->lb0_G) return fail(GPJC_EUNSUPPORTED, "the stored-matrix operator has fixed launch knobs");
  if (nchunk < 1 || nchunk > op->nchunk_max) return fail(GPJC_EINVAL, "nchunk must be in [1, %d]", op->nchunk_max);
  if (nchunk_adj < 1 || nchunk_adj > op->nchunk_a_max)
    return fail(GPJC_EINVAL, "nchunk_adj must be in [1, %d]", op->nchunk_a_max);
  if (adj_pieces < 1 || adj_pieces > kMaxAdjPieces) return fail(GPJC_EINVAL, "adj_pieces must be in [1, %d]", kMaxAdjPieces);
  op->nchunk = nchunk;
  op->nchunk_a = nchunk_adj;
  op->adj_pieces = adj_pieces;
  if (op->gexec) {
    cudaGraphExecDestroy(op->gexec);
    op->gexec = nullptr;
    op->gkey.clear();
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_op_autotune(gpjc_op* op, void* stream, int32_t* nchunk_out) {
  if (!op) return fail(GPJC_EINVAL, "null operator");
  if (op->lb0_G) {  // stored-matrix operator: one forward plane, fixed adjoint split
    if (nchunk_out) *nchunk_out = op->nchunk;
    return GPJC_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int keep_f = op->nchunk, keep_a = op->nchunk_a, keep_p = op->adj_pieces;
  gpjc_status s = GPJC_OK;
  // adjoint chunks first (forward fixed), then forward chunks, then (16-bit
  // operators) the row pieces of the adjoint
  const int npass = op->tc_ro ? 3 : 2;
  for (int pass = 0; pass < npass && !s; ++pass) {
    if (pass == 1 && fwd_balanced(op)) continue;  // the forward chunk count is not used
    int* knob = pass == 0 ? &op->nchunk_a : pass == 1 ? &op->nchunk : &op->adj_pieces;
    const int nmax = pass == 0 ? op->nchunk_a_max : pass == 1 ? op->nchunk_max : kMaxAdjPieces;
    float best = 1e30f;
    int best_n = *knob;
    // coil-chunk candidates beyond powers of two: the grid is rows x chunks
    // blocks, and a count that fills the last wave of resident blocks better
    // can win (2d256 adjoint: 6 chunks 188 us, 8 chunks 197 us); chunk counts
    // that would leave a chunk empty are skipped
    static const int kCand[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32};
    for (int ci = 0; ci < (int)(sizeof(kCand) / sizeof(kCand[0])) && !s; ++ci) {
      const int n = kCand[ci];
      if (n > nmax) break;
      if (pass < 2 && n == 7) continue;  // chunk counts: 1-6, 8, 10, ...; row pieces: 1-8
      if (pass < 2) {
        const int cpc = (op->plan->nc + n - 1) / n;
        if ((n - 1) * cpc >= op->plan->nc) continue;
      }
      *knob = n;
      float ms = 0.f;
      if ((s = time_normal(op, st, e0, e1, &ms))) break;
      if (ms < best) {
        best = ms;
        best_n = n;
      }
    }
    *knob = best_n;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) {
    op->nchunk = keep_f;
    op->nchunk_a = keep_a;
    op->adj_pieces = keep_p;
    return s;
  }
  if (op->gexec) {
    cudaGraphExecDestroy(op->gexec);
    op->gexec = nullptr;
    op->gkey.clear();
  }
  if (nchunk_out) *nchunk_out = op->nchunk;
  return GPJC_OK;
}

// ------------------------------------------------------------------ recon --
static gpjc_status recon_body(gpjc_op* op, const float2* Sc, float2* x, const gpjc_recon_params& rp,
                              cudaStream_t st) {
  const Geo& g = op->plan->geo;
  const size_t L = op->L;
  double* sc = op->sc;
  gpjc_status s;
  op->prof_used = 0;
  op->prof_marks.clear();
  CK(cudaMemsetAsync(op->status, 0, sizeof(int), st));
  // b = E_c^H S'
  if ((s = op_adj_parts(op, Sc, st))) return s;
  CK(launch_sum_parts(op->xparts, op->nchunk_a, L, op->vb, op->partials, op->counter, sc + SC_BB, st));
  if (rp.alg == GPJC_CG) {
    if (rp.use_x0) {
      if ((s = op_normal_parts(op, x, nullptr, st))) return s;
      CK(launch_sum_parts(op->xparts, op->nchunk_a, L, op->vtmp, nullptr, nullptr, nullptr, st));
      CK(launch_axpby(op->vr, op->vb, op->vtmp, 1.0f, -1.0f, L, st));
    } else {
      CK(launch_zero(x, L, st));
      CK(launch_copy(op->vr, op->vb, L, st));
    }
    CK(launch_sum_parts(op->vr, 1, L, op->vp, op->partials, op->counter, sc + SC_RR0, st));
    CK(cudaMemcpyAsync(op->hist, sc + SC_RR0, sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < rp.iters; ++it) {
      double* rr = sc + (it % 2 ? SC_RR1 : SC_RR0);
      double* rrn = sc + (it % 2 ? SC_RR0 : SC_RR1);
      if ((s = op_normal_parts(op, op->vp, sc + SC_QQ, st))) return s;
      double* h = (it + 1 < op->hist_len) ? op->hist + it + 1 : nullptr;
      CK(launch_cg_update1(op->xparts, op->nchunk_a, L, x, op->vr, op->vp, rr, sc + SC_QQ, op->partials, op->counter,
                           rrn, h, op->status, st));
      CK(launch_cg_update2(op->vp, op->vr, L, rr, rrn, st));
    }
    return GPJC_OK;
  }
  if (rp.alg == GPJC_DECOUPLED) {
    // hybrid-space reconstruction (Sec. 3.4, algorithm #1): CG with the
    // scalars of each aliased set (b = E_c^H S' is steps 1 and the first
    // half of 2: the phase-encode adjoint gives h~, the readout adjoint G^H)
    const gpjc_plan* pl = op->plan;
    const int ns = pl->n_sets;
    double* rowval = op->ds_rowval;
    double* rrs[2] = {op->ds_sc, op->ds_sc + ns};
    double* pap = op->ds_sc + 2 * ns;
    if (rp.use_x0) {
      if ((s = op_normal_parts(op, x, nullptr, st))) return s;
      CK(launch_sum_parts(op->xparts, op->nchunk_a, L, op->vtmp, nullptr, nullptr, nullptr, st));
      CK(launch_axpby(op->vr, op->vb, op->vtmp, 1.0f, -1.0f, L, st));
    } else {
      CK(launch_zero(x, L, st));
      CK(launch_copy(op->vr, op->vb, L, st));
    }
    CK(launch_copy(op->vp, op->vr, L, st));
    CK(launch_ds_rowdot(op->vr, 1, L, g.rows, g.nx, nullptr, nullptr, rowval, st));
    CK(launch_ds_setsum(rowval, pl->d_set_ptr, pl->d_set_rows, ns, rrs[0], op->hist, st));
    for (int it = 0; it < rp.iters; ++it) {
      double* rr = rrs[it % 2];
      double* rrn = rrs[(it + 1) % 2];
      if ((s = op_normal_parts(op, op->vp, nullptr, st))) return s;
      // q = N p (into vtmp) and <p, q> per set
      CK(launch_ds_rowdot(op->xparts, op->nchunk_a, L, g.rows, g.nx, op->vtmp, op->vp, rowval, st));
      CK(launch_ds_setsum(rowval, pl->d_set_ptr, pl->d_set_rows, ns, pap, nullptr, st));
      CK(launch_ds_update1(g.rows, g.nx, pl->d_set_of_row, x, op->vr, op->vp, op->vtmp, rr, pap, rowval, op->status,
                           st));
      double* h = (it + 1 < op->hist_len) ? op->hist + it + 1 : nullptr;
      CK(launch_ds_setsum(rowval, pl->d_set_ptr, pl->d_set_rows, ns, rrn, h, st));
      CK(launch_ds_update2(g.rows, g.nx, pl->d_set_of_row, op->vp, op->vr, rr, rrn, st));
    }
    return GPJC_OK;
  }
  // FISTA
  if (rp.lipschitz > 0.0) {
    CK(launch_set_scalar(sc + SC_LIP, rp.lipschitz, st));
  } else {
    const int pit = rp.power_iters > 0 ? rp.power_iters : 20;
    CK(launch_scale_by(op->vv, op->vb, sc + SC_BB, L, nullptr, st));
    for (int it = 0; it < pit; ++it) {
      if ((s = op_normal_parts(op, op->vv, nullptr, st))) return s;
      CK(launch_sum_parts(op->xparts, op->nchunk_a, L, op->vtmp, op->partials, op->counter, sc + SC_NV, st));
      CK(launch_scale_by(op->vv, op->vtmp, sc + SC_NV, L, sc + SC_LIP, st));
    }
    // the smoothed TV gradient is Lipschitz with constant ||D||^2 / eps <= 8 / eps
    if (rp.lambda_tv > 0.0) CK(launch_add_scalar(sc + SC_LIP, 8.0 * rp.lambda_tv / rp.tv_eps, st));
  }
  if (!rp.use_x0) CK(launch_zero(x, L, st));
  CK(launch_copy(op->vy, x, L, st));
  const bool tv = rp.lambda_tv > 0.0;
  double t = 1.0;
  for (int it = 0; it < rp.iters; ++it) {
    if ((s = op_normal_parts(op, op->vy, nullptr, st))) return s;
    if (tv) CK(launch_tv_grad(op->vy, op->vtmp, g.nz, g.ny, g.nx, (float)(rp.tv_eps * rp.tv_eps), st));
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    const double ck = (t - 1.0) / tn;
    CK(launch_fista_step(g, op->xparts, op->nchunk_a, x, op->vy, op->vb, sc + SC_LIP, rp.lambda, rp.haar_levels, ck,
                         tv ? op->vtmp : nullptr, rp.lambda_tv, op->status, st));
    t = tn;
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_recon(const gpjc_op* cop, const float* d_Sc, float* d_x, const gpjc_recon_params* params,
                                  gpjc_recon_info* info, void* stream) {
  if (!cop || !d_Sc || !d_x || !params) return fail(GPJC_EINVAL, "null argument");
  gpjc_op* op = const_cast<gpjc_op*>(cop);
  const gpjc_recon_params rp = *params;
  const Geo& g = op->plan->geo;
  if (rp.alg != GPJC_CG && rp.alg != GPJC_FISTA && rp.alg != GPJC_DECOUPLED)
    return fail(GPJC_EINVAL, "unknown algorithm");
  if (rp.iters < 0 || rp.iters > 100000) return fail(GPJC_EINVAL, "iters out of range");
  if (rp.alg == GPJC_FISTA) {
    if (rp.haar_levels < 0 || rp.haar_levels > 5) return fail(GPJC_EINVAL, "haar_levels must be in [0, 5]");
    const int ts = 1 << rp.haar_levels;
    if (g.nx % ts || g.ny % ts) return fail(GPJC_EINVAL, "nx, ny must be divisible by 2^haar_levels");
    if (!(rp.lambda >= 0.0) || !std::isfinite(rp.lambda)) return fail(GPJC_EINVAL, "lambda must be finite and >= 0");
    if (!std::isfinite(rp.lipschitz)) return fail(GPJC_EINVAL, "lipschitz must be finite");
    if (!(rp.lambda_tv >= 0.0) || !std::isfinite(rp.lambda_tv))
      return fail(GPJC_EINVAL, "lambda_tv must be finite and >= 0");
    if (rp.lambda_tv > 0.0) {
      const double e2 = rp.tv_eps * rp.tv_eps;
      if (!(rp.tv_eps > 0.0) || !(e2 >= (double)FLT_MIN) || !(e2 <= (double)FLT_MAX))
        return fail(GPJC_EINVAL, "tv_eps must be > 0 with tv_eps^2 a normal FP32 number");
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  gpjc_status s;
  if (rp.use_graph) {
    std::vector<char> key(sizeof(rp) + 2 * sizeof(void*) + 3 * sizeof(int));
    memcpy(key.data(), &rp, sizeof(rp));
    memcpy(key.data() + sizeof(rp), &d_Sc, sizeof(void*));
    memcpy(key.data() + sizeof(rp) + sizeof(void*), &d_x, sizeof(void*));
    memcpy(key.data() + sizeof(rp) + 2 * sizeof(void*), &op->nchunk, sizeof(int));
    memcpy(key.data() + sizeof(rp) + 2 * sizeof(void*) + sizeof(int), &op->nchunk_a, sizeof(int));
    memcpy(key.data() + sizeof(rp) + 2 * sizeof(void*) + 2 * sizeof(int), &op->adj_pieces, sizeof(int));
    cudaStream_t cs = op->cap_st;
    CK(cudaEventRecord(op->ev_in, st));
    CK(cudaStreamWaitEvent(cs, op->ev_in, 0));
    if (!op->gexec || key != op->gkey) {
      if (op->gexec) {
        cudaGraphExecDestroy(op->gexec);
        op->gexec = nullptr;
        op->gkey.clear();
      }
      // one eager pass sets every kernel attribute outside the capture and
      // produces the result of this call
      if ((s = recon_body(op, (const float2*)d_Sc, (float2*)d_x, rp, cs))) return s;
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
      g_capturing = true;
      s = recon_body(op, (const float2*)d_Sc, (float2*)d_x, rp, cs);
      g_capturing = false;
      cudaError_t ce = cudaStreamEndCapture(cs, &graph);
      if (s) return s;
      if (ce != cudaSuccess) return fail(GPJC_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
      {
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
        int kn = 0;
        for (auto nd : nodes) {
          cudaGraphNodeType ty;
          if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kn;
        }
        op->graph_kernels = kn;
      }
      ce = cudaGraphInstantiate(&op->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return fail(GPJC_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
      op->gkey = key;
    } else {
      CK(cudaGraphLaunch(op->gexec, cs));
      note_launches(op->graph_kernels);
    }
    CK(cudaEventRecord(op->ev_out, cs));
    CK(cudaStreamWaitEvent(st, op->ev_out, 0));
  } else {
    if ((s = recon_body(op, (const float2*)d_Sc, (float2*)d_x, rp, st))) return s;
  }
  if (info) {
    int dev_status = 0;
    double lip = 0.0;
    CK(cudaMemcpyAsync(&dev_status, op->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&lip, op->sc + SC_LIP, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (info->h_history && rp.alg == GPJC_CG) {
      const int n = std::min(rp.iters + 1, op->hist_len);
      CK(cudaMemcpyAsync(info->h_history, op->hist, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    info->status = dev_status == kDevNonFinite ? GPJC_ENONFINITE : (dev_status ? GPJC_ETIMEOUT : GPJC_OK);
    info->lipschitz = lip;
    if (dev_status) return fail((gpjc_status)info->status, "device status %d", dev_status);
  }
  return GPJC_OK;
}

// ------------------------------------------------------------------ profiling --
extern "C" gpjc_status gpjc_op_profile(gpjc_op* op, int32_t enable) {
  if (!op) return fail(GPJC_EINVAL, "null operator");
  if (enable && op->prof_pool.empty()) {
    op->prof_pool.resize(8192);
    for (auto& e : op->prof_pool) CK(cudaEventCreate(&e));
  }
  op->prof_on = enable != 0;
  op->prof_used = 0;
  op->prof_marks.clear();
  if (op->gexec) {  // the cached graph was captured with the other setting
    cudaGraphExecDestroy(op->gexec);
    op->gexec = nullptr;
    op->gkey.clear();
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_op_profile_read(const gpjc_op* op, int32_t stage, double* total_ms, int32_t* count) {
  if (!op || !total_ms || !count) return fail(GPJC_EINVAL, "null argument");
  double tot = 0.0;
  int n = 0;
  for (const auto& mk : op->prof_marks) {
    if (mk.first != stage) continue;
    CK(cudaEventSynchronize(op->prof_pool[mk.second + 1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, op->prof_pool[mk.second], op->prof_pool[mk.second + 1]));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *count = n;
  return GPJC_OK;
}

// ------------------------------------------------------------------ no-allocation adjoint --
// A variant of gpjc_apply_EH whose scratch (the hybrid matrix, and in 3D the
// phase-encode intermediate) lives in a fixed device array of this library
// instead of an operator workspace, so a call allocates nothing.
static constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
static std::mutex g_static_mu;
// per device ordinal: the context the address was looked up in, and the
// address (looked up again when the device's context changed, e.g. after
// cudaDeviceReset)
static void* g_static_ctx[256];
static void* g_static_addr[256];

// current driver context, through the runtime's driver entry-point lookup
// (nullptr when unavailable)
static void* current_context() {
  using ctx_fn = int (*)(void**);
  static ctx_fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (ctx_fn)f;
  }
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

// true when `p` is device (or managed) memory of device `dev`
static bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

extern "C" gpjc_status gpjc_apply_EH_static(const gpjc_groups* gr, const float* d_coil, const float* d_y,
                                            float* d_x, void* stream) {
  if (!gr || !d_coil || !d_y || !d_x) return fail(GPJC_EINVAL, "null argument");
  const Geo& g = gr->plan->geo;
  const size_t hybrid = sizeof(float2) * (size_t)g.rows * g.ntxc;
  const size_t need = g.dim3d ? 2 * hybrid : hybrid;
  if (need > kStaticScratchBytes)
    return fail(GPJC_EINVAL, "gpjc_apply_EH_static needs %zu bytes of scratch; its static scratch holds %zu",
                need, kStaticScratchBytes);
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(GPJC_EUNSUPPORTED, "device ordinal %d out of range", dev);
  // the kernels run on the current device: every buffer must live there
  if (!on_device(d_coil, dev) || !on_device(d_y, dev) || !on_device(d_x, dev))
    return fail(GPJC_EINVAL, "d_coil, d_y and d_x must be device memory of the current device (%d)", dev);
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    void* ctx = current_context();
    if (!g_static_addr[dev] || g_static_ctx[dev] != ctx) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p)
        return fail(GPJC_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
      g_static_addr[dev] = p;
      g_static_ctx[dev] = ctx;
    }
    base = g_static_addr[dev];
  }
  float2* H2 = (float2*)base;
  float2* T = g.dim3d ? H2 + (size_t)g.rows * g.ntxc : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  // H2 and T are fully overwritten before they are read: nothing to clear.
  CK(launch_pe_adj(g, (const float2*)d_y, g.ntxc, T, H2, st));
  CK(launch_k1_adj_fp32(g, H2, (const float2*)d_coil, gr->A, (float2*)d_x, 1, st));
  return GPJC_OK;
}

// ------------------------------------------------------------------ batched CG --
struct gpjc_batch {
  int n, iters, n_stages, grid;
  long long wait_cycles;
  size_t smem;
  std::vector<gpjc_op*> ops;
  std::vector<BatchSlice> hs;      // host copy of the slice descriptors
  std::vector<long long> stage_start;
  std::vector<int> slice_off;
  BatchSlice* d_slices;
  long long* d_stage_start;
  int* d_slice_off;
  int* d_done;
  unsigned long long* d_head;
  int* d_abort;
  int* d_status;
  double* d_scal;                  // [n][2 iters + 1]
  cudaGraphExec_t gexec;
  std::vector<const void*> gkey;
  DevMem mem;
};

extern "C" gpjc_status gpjc_batch_create(int32_t n, gpjc_op* const* ops, int32_t iters, gpjc_batch** out) {
  if (!ops || !out || n < 1) return fail(GPJC_EINVAL, "need at least one operator");
  if (iters < 0 || iters > 10000) return fail(GPJC_EINVAL, "iters out of range");
  *out = nullptr;
  auto* b = new (std::nothrow) gpjc_batch();
  if (!b) return fail(GPJC_ENOMEM, "host allocation");
  std::unique_ptr<gpjc_batch> guard(b);
  b->n = n;
  b->iters = iters;
  b->n_stages = 3 + 5 * iters;
  b->ops.assign(ops, ops + n);
  b->hs.resize(n);
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    gpjc_op* op = ops[i];
    if (!op) return fail(GPJC_EINVAL, "operator %d is null", i);
    const gpjc_plan* p = op->plan;
    const Geo& g = p->geo;
    if (op->prec != GPJC_FP32) return fail(GPJC_EUNSUPPORTED, "batched CG runs the FP32 operator (slice %d)", i);
    if (g.dim3d) return fail(GPJC_EUNSUPPORTED, "batched CG is 2D (slice %d)", i);
    if (!p->rt_f.rb || !p->rt_a.rb || p->rt_f.nt > 512)
      return fail(GPJC_EUNSUPPORTED, "slice %d has no register-tile plan for the batch kernel", i);
    for (int j = 0; j < i; ++j)
      if (ops[j] == op) return fail(GPJC_EINVAL, "operator %d appears twice", i);
    BatchSlice& s = b->hs[i];
    memset(&s, 0, sizeof s);
    s.g = g;
    s.rtf = p->rt_f;
    s.rta = p->rt_a;
    s.nchunk = op->nchunk;
    s.cpc = (g.nc + op->nchunk - 1) / op->nchunk;
    s.n_f = ((g.rows + p->rt_f.rb - 1) / p->rt_f.rb) * op->nchunk;
    s.n_a = ((g.rows + p->rt_a.rb - 1) / p->rt_a.rb) * op->nchunk;
    s.n_pe = (g.ntxc + kPeCBHost - 1) / kPeCBHost;
    s.n_vec = (int)((op->L + kVecChunkHost - 1) / kVecChunkHost);
    s.mt_f = (p->rt_f.nt + 255) / 256;
    const int mx = (p->rt_a.rb * g.nx + 255) / 256;
    s.mx_a = mx <= 1 ? 1 : mx <= 2 ? 2 : mx <= 4 ? 4 : 8;
    if (p->rt_a.ts == 2) s.mx_a = mx <= 1 ? 5 : 6;  // two-sample tiles (one row per block)
    if (mx > 8) return fail(GPJC_EUNSUPPORTED, "slice %d: adjoint rows too wide", i);
    s.coil = op->coil;
    s.AT = op->gr->AT;
    s.A = op->gr->A;
    s.Hpart = op->Hpart;
    s.H2 = op->H2;
    s.xparts = op->xparts;
    s.r = op->vr;
    s.p = op->vp;
    smem = std::max(smem, std::max(readout_fwd_smem(g, p->rt_f.rb), readout_adj_smem(g, p->rt_a.rb, p->rt_a.hstage)));
    smem = std::max(smem, batch_pe_smem(g));
  }
  b->smem = smem;
  // queue layout: stage-major, then slice, then item
  const int types = 7;
  b->slice_off.assign((size_t)types * (n + 1), 0);
  for (int t = 0; t < types; ++t)
    for (int i = 0; i < n; ++i) {
      const BatchSlice& s = b->hs[i];
      const int items = (t == 0 || t == 4) ? s.n_pe : (t == 1) ? s.n_a : (t == 3) ? s.n_f : s.n_vec;
      b->slice_off[(size_t)t * (n + 1) + i + 1] = b->slice_off[(size_t)t * (n + 1) + i] + items;
    }
  b->stage_start.assign(b->n_stages + 1, 0);
  for (int j = 0; j < b->n_stages; ++j) {
    int t = j < 3 ? j : ((j - 3) % 5 == 0 ? 3 : (j - 3) % 5 == 1 ? 4 : (j - 3) % 5 == 2 ? 1 : (j - 3) % 5 == 3 ? 5 : 6);
    b->stage_start[j + 1] = b->stage_start[j] + b->slice_off[(size_t)t * (n + 1) + n];
  }
  DevMem& m = b->mem;
  gpjc_status s;
  if ((s = m.alloc(&b->d_slices, n)) || (s = m.upload(&b->d_stage_start, b->stage_start)) ||
      (s = m.upload(&b->d_slice_off, b->slice_off)) || (s = m.alloc(&b->d_done, (size_t)n * b->n_stages)) ||
      (s = m.alloc(&b->d_head, 1)) || (s = m.alloc(&b->d_abort, 1)) || (s = m.alloc(&b->d_status, 1)) ||
      (s = m.alloc(&b->d_scal, (size_t)n * (2 * iters + 1))))
    return s;
  for (int i = 0; i < n; ++i) {
    b->hs[i].rr = b->d_scal + (size_t)i * (2 * iters + 1);
    b->hs[i].qq = b->hs[i].rr + iters + 1;
  }
  b->wait_cycles = 4000000000ll;  // about 2 s at the maximum SM clock
  b->grid = batch_max_blocks(smem);
  if (b->grid < 1) return fail(GPJC_EUNSUPPORTED, "batch kernel does not fit on an SM (%zu B shared memory)", smem);
  b->gexec = nullptr;
  *out = guard.release();
  return GPJC_OK;
}

extern "C" void gpjc_batch_destroy(gpjc_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  delete b;
}

static gpjc_status batch_body(gpjc_batch* b, cudaStream_t st) {
  const int n = b->n;
  CK(cudaMemsetAsync(b->d_done, 0, sizeof(int) * (size_t)n * b->n_stages, st));
  CK(cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(b->d_abort, 0, sizeof(int), st));
  CK(cudaMemsetAsync(b->d_status, 0, sizeof(int), st));
  CK(cudaMemsetAsync(b->d_scal, 0, sizeof(double) * (size_t)n * (2 * b->iters + 1), st));
  BatchPlan bp;
  bp.n_slices = n;
  bp.n_stages = b->n_stages;
  bp.slices = b->d_slices;
  bp.stage_start = b->d_stage_start;
  bp.slice_off = b->d_slice_off;
  bp.done = b->d_done;
  bp.head = b->d_head;
  bp.abort = b->d_abort;
  bp.status = b->d_status;
  bp.wait_cycles = b->wait_cycles;
  CK(launch_batch_cg(bp, b->grid, b->smem, st));
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_recon_batched(gpjc_batch* b, const float* const* d_Sc, float* const* d_x,
                                          int32_t use_graph, int32_t* h_status, void* stream) {
  if (!b || !d_Sc || !d_x) return fail(GPJC_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<const void*> key(2 * b->n);
  for (int i = 0; i < b->n; ++i) {
    if (!d_Sc[i] || !d_x[i]) return fail(GPJC_EINVAL, "slice %d: null data pointer", i);
    key[2 * i] = d_Sc[i];
    key[2 * i + 1] = d_x[i];
  }
  const bool same = (key == b->gkey);
  if (!same) {
    for (int i = 0; i < b->n; ++i) {
      b->hs[i].Sc = (const float2*)d_Sc[i];
      b->hs[i].x = (float2*)d_x[i];
    }
    CK(cudaMemcpy(b->d_slices, b->hs.data(), sizeof(BatchSlice) * b->n, cudaMemcpyHostToDevice));
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    b->gkey = key;
  }
  gpjc_status s;
  if (use_graph) {
    if (!b->gexec) {
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t graph;
      cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
      if (ce == cudaSuccess) {
        g_capturing = true;
        s = batch_body(b, cs);
        g_capturing = false;
        ce = cudaStreamEndCapture(cs, &graph);
        if (!s && ce == cudaSuccess) {
          ce = cudaGraphInstantiate(&b->gexec, graph, 0);
          cudaGraphDestroy(graph);
        }
      }
      cudaStreamDestroy(cs);
      if (s) return s;
      if (ce != cudaSuccess) return fail(GPJC_ECUDA, "batch graph: %s", cudaGetErrorString(ce));
    }
    CK(cudaGraphLaunch(b->gexec, st));
    note_launches(1);
  } else {
    if ((s = batch_body(b, st))) return s;
  }
  if (h_status) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *h_status = v == kDevNonFinite ? GPJC_ENONFINITE : (v ? GPJC_ETIMEOUT : GPJC_OK);
    if (v) return fail((gpjc_status)*h_status, "batched reconstruction device status %d", v);
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_batch_set_wait_budget(gpjc_batch* b, int64_t cycles) {
  if (!b || cycles < 0) return fail(GPJC_EINVAL, "invalid argument");
  b->wait_cycles = cycles;
  if (b->gexec) {  // the budget is a kernel argument of the captured graph
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return GPJC_OK;
}

extern "C" gpjc_status gpjc_batch_info(const gpjc_batch* b, int32_t* grid, int64_t* items) {
  if (!b) return fail(GPJC_EINVAL, "null batch");
  if (grid) *grid = b->grid;
  if (items) *items = b->stage_start.back();
  return GPJC_OK;
}

// ------------------------------------------------------------------ multi-slice graph --
// Many reconstructions (any operators: sizes, coil counts, precisions, 2D or
// 3D, any algorithm) captured together in one CUDA graph whose slices run on
// parallel branches: each branch runs its slices' reconstructions one after
// another with the single-slice kernels, and the branches share the GPU, so
// the launch gaps, small grids and tails of one slice are filled by the
// others.  Slices are assigned longest first to the least-loaded branch
// (cost: readout work rows x coils x N_tx).
struct gpjc_multi {
  int n, nb;
  std::vector<gpjc_op*> ops;
  std::vector<std::vector<int>> branch;  // slices of each branch, in order
  std::vector<cudaStream_t> streams;     // one per branch
  std::vector<cudaEvent_t> join;         // one per branch
  cudaStream_t cs;
  cudaEvent_t fork;
  cudaGraphExec_t gexec;
  std::vector<char> gkey;
  int* d_status;                         // gathered per-slice status words
  DevMem mem;
  ~gpjc_multi() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto s : streams) cudaStreamDestroy(s);
    for (auto e : join) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
    if (fork) cudaEventDestroy(fork);
  }
};

extern "C" gpjc_status gpjc_multi_create(int32_t n, gpjc_op* const* ops, int32_t n_branches, gpjc_multi** out) {
  if (!ops || !out || n < 1) return fail(GPJC_EINVAL, "need at least one operator");
  if (n_branches < 1 || n_branches > 64) return fail(GPJC_EINVAL, "n_branches must be in [1, 64]");
  *out = nullptr;
  auto* m = new (std::nothrow) gpjc_multi();
  if (!m) return fail(GPJC_ENOMEM, "host allocation");
  m->cs = nullptr;
  m->fork = nullptr;
  m->gexec = nullptr;
  std::unique_ptr<gpjc_multi> guard(m);
  m->n = n;
  m->nb = std::min<int>(n_branches, n);
  m->ops.assign(ops, ops + n);
  for (int i = 0; i < n; ++i) {
    if (!ops[i]) return fail(GPJC_EINVAL, "operator %d is null", i);
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) return fail(GPJC_EINVAL, "operator %d appears twice (its workspaces would race)", i);
  }
  // longest first onto the least-loaded branch
  std::vector<std::pair<double, int>> cost(n);
  for (int i = 0; i < n; ++i) {
    const Geo& g = ops[i]->plan->geo;
    cost[i] = {(double)g.rows * g.nc * g.ntx, i};
  }
  std::stable_sort(cost.begin(), cost.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  m->branch.assign(m->nb, {});
  std::vector<double> load(m->nb, 0.0);
  for (const auto& c : cost) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    m->branch[k].push_back(c.second);
    load[k] += c.first;
  }
  m->streams.assign(m->nb, nullptr);
  m->join.assign(m->nb, nullptr);
  for (int k = 0; k < m->nb; ++k) {
    CK(cudaStreamCreateWithFlags(&m->streams[k], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&m->join[k], cudaEventDisableTiming));
  }
  CK(cudaStreamCreateWithFlags(&m->cs, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming));
  gpjc_status s;
  if ((s = m->mem.alloc(&m->d_status, (size_t)n))) return s;
  *out = guard.release();
  return GPJC_OK;
}

extern "C" void gpjc_multi_destroy(gpjc_multi* m) { delete m; }

extern "C" gpjc_status gpjc_recon_multi(gpjc_multi* m, const float* const* d_Sc, float* const* d_x,
                                        const gpjc_recon_params* params, int32_t* h_status, void* stream) {
  if (!m || !d_Sc || !d_x || !params) return fail(GPJC_EINVAL, "null argument");
  gpjc_recon_params rp = *params;
  rp.use_x0 = 0;
  rp.use_graph = 0;
  if (rp.alg != GPJC_CG && rp.alg != GPJC_DECOUPLED)
    return fail(GPJC_EUNSUPPORTED, "the multi-slice graph runs CG or the decoupled CG");
  if (rp.iters < 0 || rp.iters > 100000) return fail(GPJC_EINVAL, "iters out of range");
  std::vector<char> key(sizeof(rp) + 2 * sizeof(void*) * m->n);
  memcpy(key.data(), &rp, sizeof(rp));
  for (int i = 0; i < m->n; ++i) {
    if (!d_Sc[i] || !d_x[i]) return fail(GPJC_EINVAL, "slice %d: null data pointer", i);
    memcpy(key.data() + sizeof(rp) + 2 * sizeof(void*) * i, &d_Sc[i], sizeof(void*));
    memcpy(key.data() + sizeof(rp) + 2 * sizeof(void*) * i + sizeof(void*), &d_x[i], sizeof(void*));
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (!m->gexec || key != m->gkey) {
    if (m->gexec) {
      cudaGraphExecDestroy(m->gexec);
      m->gexec = nullptr;
    }
    // every kernel attribute is set outside the capture by one eager pass of
    // each slice (its result is overwritten by the graph launch below)
    for (int i = 0; i < m->n; ++i) {
      gpjc_status s = recon_body(m->ops[i], (const float2*)d_Sc[i], (float2*)d_x[i], rp, m->cs);
      if (s) return s;
    }
    CK(cudaStreamSynchronize(m->cs));
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(m->cs, cudaStreamCaptureModeRelaxed));
    g_capturing = true;
    gpjc_status s = GPJC_OK;
    cudaError_t ce = cudaEventRecord(m->fork, m->cs);
    for (int k = 0; k < m->nb && ce == cudaSuccess && !s; ++k) {
      ce = cudaStreamWaitEvent(m->streams[k], m->fork, 0);
      for (int i : m->branch[k]) {
        if (ce != cudaSuccess || s) break;
        s = recon_body(m->ops[i], (const float2*)d_Sc[i], (float2*)d_x[i], rp, m->streams[k]);
        if (!s) ce = cudaMemcpyAsync(m->d_status + i, m->ops[i]->status, sizeof(int), cudaMemcpyDeviceToDevice,
                                     m->streams[k]);
      }
      if (ce == cudaSuccess) ce = cudaEventRecord(m->join[k], m->streams[k]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(m->cs, m->join[k], 0);
    }
    g_capturing = false;
    const cudaError_t ee = cudaStreamEndCapture(m->cs, &graph);
    if (s) {
      if (ee == cudaSuccess) cudaGraphDestroy(graph);
      return s;
    }
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (ee == cudaSuccess) cudaGraphDestroy(graph);
      return fail(GPJC_ECUDA, "multi-slice graph capture: %s",
                  cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    ce = cudaGraphInstantiate(&m->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(GPJC_ECUDA, "multi-slice graph: %s", cudaGetErrorString(ce));
    m->gkey = key;
  }
  CK(cudaGraphLaunch(m->gexec, st));
  note_launches(1);
  if (h_status) {
    std::vector<int> v(m->n, 0);
    CK(cudaMemcpyAsync(v.data(), m->d_status, sizeof(int) * m->n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int worst = 0;
    for (int i = 0; i < m->n; ++i) worst = std::max(worst, v[i]);
    *h_status = worst == kDevNonFinite ? GPJC_ENONFINITE : (worst ? GPJC_ETIMEOUT : GPJC_OK);
    if (worst) return fail((gpjc_status)*h_status, "multi-slice reconstruction device status %d", worst);
  }
  return GPJC_OK;
}
