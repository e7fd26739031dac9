// Internal structures shared by the host API (gpjc_api.cu) and the kernel
// translation units.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpjc {

constexpr int kMaxStages = 12;

// Radix plan of one FFT length (product of 2,3,4,5,7,8).
struct FftPlan {
  int n;
  int nst;
  int rad[kMaxStages];
  int n1, n2;  // two-pass plan n = n1 n2 (0 when n has none; then the radix stages run)
};

// Lengths that have a two-pass FFT plan n = n1 n2 (the list is shared by the
// host planner and the device dispatcher).
__host__ __device__ constexpr int fft2p_code(int n1, int n2) { return n1 * 64 + n2; }
__host__ __device__ constexpr bool fft2p_supported(int n1, int n2) {
  return (n1 == 16 && (n2 == 8 || n2 == 10 || n2 == 12 || n2 == 14 || n2 == 15 || n2 == 16 || n2 == 18 ||
                       n2 == 20)) ||
         (n1 == 8 && (n2 == 5 || n2 == 7));
}

// Geometry and device-resident bookkeeping tables, passed to kernels by
// value.  All pointers are device pointers owned by the plan.
struct Geo {
  int nx, ny, nz, nc, os, ntx, w, G, ns, np, ntxc, rows, n_lines, keep_max;
  int dim3d;  // nz > 1
  float inv_sqrt_ntx, inv_sqrt_ny, inv_sqrt_nz;
  FftPlan fx, fy, fz;
  const int* pg;          // [np] patch -> group
  const int* poff;        // [np] first compressed column of patch
  const int* keep;        // [G]
  const int* aoff;        // [G] offset of group g inside packed A (complex elems)
  const int* out_tbase;   // [ntxc] first readout sample of the column's patch
  const int* out_abase;   // [ntxc] aoff[g] + k for the column
  const int* out_astride; // [ntxc] keep[g] of the column's group
  const int* line_ky;     // [n_lines]
  const int* line_kz;     // [n_lines]
  const int* line_of;     // [nz*ny] line index of (kz, ky) or -1
  const float* ay;        // [ntx] wave excursion a_y(t) (phase-encode lines)
  const float* az;        // [ntx]
  const float2* tw_x;     // [nx] exp(-2 pi i k / nx)
  const float2* tw_y;     // [ny]
  const float2* tw_z;     // [nz]
  const float2* pre;      // [os * nx] (-1)^x exp(-2 pi i s x / ntx)
  const float2* post_y;   // [ny][ntx] (-1)^{m+nx/2} e^{i pi s/os} e^{-2 pi i a_y(t) y_c/ny} / sqrt(ntx)
  const float2* post_z;   // [nz][ntx] e^{-2 pi i a_z(t) z_c/nz}
};

// Register-tile tables of the readout stage (k_readout.cu).  rb rows per
// block; forward tiles: hdr = (aoff_g + k0, keep_g, kept count, 0), cols =
// (r * stride + p w, r * ntxc + off_p + k0) or (-1, -1); adjoint tiles:
// hdr = (aoff_g + tau0, keep_g, sample count, 0), cols = (r, off_p,
// p w + tau0, 0) or (-1, ...).
struct RTiles {
  int rb;
  int nt;
  int ts;            // adjoint: readout samples per tile (2 or 4)
  int hstage;        // adjoint: the block's rows of H2 are staged in shared memory (rb == 1)
  int hpair;         // adjoint, staged: paired layout (hswz) read two kept components per load
  int nb;            // forward: coils per batched-transform step of k1f_batched; 0: per-row kernel
  // forward, balanced launch of k1f_batched (bal_units > 0): one wave of
  // bal_grid blocks over bal_units (row block, coil group) units, bal_npair
  // units per row block, partial sums in bal_planes planes
  int bal_grid, bal_units, bal_npair, bal_planes;
  const int4* hdr;   // [nt]
  const int4* cols;  // [nt * 4]
};

// Tensor-core group compression geometry (k_tc.cu).  The group map must be
// periodic: patch p belongs to group p mod G and P = G w divides N_tx, so
// group g's occurrences start at g w + q P (q < n_occ).
struct TcGeom {
  int G, w, nc, ns, ntx, ntxc;
  int n_occ, P, lt;          // occurrences per readout line, period, lines per 128-column tile
  int ncc, nchunks, Kc;      // coils per K chunk, chunks, K per chunk (multiple of 16)
  int npad;                  // N of the compression GEMM: 2 keep_max rounded up to 16
  int box0, xalign;          // TMA inner box (elements) and coordinate alignment
  int stg_tx, stg_bytes;     // staging bytes per chunk (exact, allocated)
  int tmem_cols;             // TMEM columns of the compression accumulator
  int Kx, nexp;              // expansion GEMM: K = 2 keep_max rounded to 16, N = 2 N_s rounded to 16
  const int* keep;
  const int* aoff;
  const int* poff;
  const float* scale;
};

// One slice of a batched persistent CG reconstruction (k_readout.cu).
struct BatchSlice {
  Geo g;
  RTiles rtf, rta;
  int nchunk, cpc;
  int n_f, n_a, n_pe, n_vec;  // items per stage type
  int mt_f, mx_a;             // register-tile variants of the readout bodies
  const float2* coil;
  const float2* AT;
  const float2* A;
  const float2* Sc;
  float2 *Hpart, *H2, *xparts, *x, *r, *p;
  double* rr;  // [iters + 1] ||r||^2 per iteration
  double* qq;  // [iters] ||E_c p||^2 per iteration
};
struct BatchPlan {
  int n_slices, n_stages;
  const BatchSlice* slices;
  const long long* stage_start;  // [n_stages + 1] first queue item of each stage
  const int* slice_off;          // [7][n_slices + 1] first item of each slice within a stage of a type
  int* done;                     // [n_slices][n_stages] completed items
  unsigned long long* head;      // next queue item
  int* abort;
  int* status;
  long long wait_cycles;         // budget of one dependency wait (SM clock cycles)
};

// Device status word values (written by kernels, read by the host).
enum DevStatus : int { kDevOk = 0, kDevNonFinite = 1, kDevTimeout = 2, kDevBadIndex = 3 };

// Count of kernels launched by this library (for launch accounting); the
// launchers add to it unless the calling thread is capturing a graph.
void note_launches(int n);

// Shared-memory budget of one k1 block (readout stage) for a geometry.
inline size_t k1_smem_bytes(const Geo& g) {
  return sizeof(float2) * (size_t)(4 * g.ntx + g.nx);
}

}  // namespace gpjc
