/*
 * gpjc — group-patch joint compression of B0/RF-encoded MRI on one GPU.
 *
 * C ABI of the compression and reconstruction hot path of
 *   R. Tian, K. Scheffler, "Group-Patch Joint Compression: Compressing Dynamic
 *   B0 and Static RF Spatial Modulations Across k-Space Subregion Groups for
 *   Highly Accelerated MRI", arXiv 2601.05418.
 *
 * Model (Sec. 2.2, Eq. 1-4):   S = E rho,  S[line][coil][t]
 *   E = M F_pe Psi F_ro C : coil multiply C, centred zero-padded readout DFT
 *   F_ro (N_tx = os N_x samples), wave phase Psi = exp(-i phi(t,y,z)) with
 *   phi = 2 pi [a_y(t) y_c/N_y + a_z(t) z_c/N_z], a_y = kappa_y (1-cos th)/2,
 *   a_z = kappa_z sin(th)/2, th = 2 pi cycles t / N_tx (Eq. 3, sinusoidal G_y,
 *   cosine G_z), centred phase-encode DFT F_pe and sampled-line gather M.
 * Compression (Sec. 2.4, Eq. 6-15): the readout is cut into patches of w
 *   samples; patch p belongs to group g = patch_group[p]; with
 *   N_s = N_C w and patch vector index i = n w + tau (coil-major),
 *   P_g = sum_{r in ROI} E_g[r] E_g[r]^H / (E_g[r]^H E_g[r])  (Eq. 7-11),
 *   P_g = U_g F_g U_g^H  (Eq. 8),  A_g = C_g U_g^H (T (x) I_w)  (Eq. 12),
 *   S'_{l,p} = A_{g(p)} s_{l,p}  (Eq. 13),  E_c = A E  (Eq. 14-15),
 *   compressed readout length N'_tx = sum_p keep[g(p)].
 * Reconstruction (Sec. 3.4): CG on E_c^H E_c x = E_c^H S' (Eq. 16), the
 *   decoupled least squares of algorithm #1 (one CG per aliased set of rows),
 *   and FISTA with an orthonormal Haar l1 term on the detail bands plus an
 *   optional smoothed isotropic TV term (Eq. 17).
 *
 * Conventions for every call:
 *   - complex data are interleaved float pairs (complex64, `float` re, im);
 *   - "d_" pointers are device memory, "h_" pointers host memory; all of them
 *     stay owned by the caller, the library never frees caller memory;
 *   - images are [nz][ny][nx] (x fastest); coil maps [nc][nz][ny][nx];
 *     raw data [n_lines][nc][ntx]; compressed data [n_lines][ntx_c];
 *   - `stream` is a cudaStream_t (NULL = legacy default stream); calls are
 *     asynchronous on it unless stated otherwise;
 *   - every call returns a gpjc_status; arguments are validated before any
 *     launch; gpjc_last_error() gives a message for the calling thread.
 *     Nothing aborts, exits or throws across the ABI.
 *   - handles are immutable after creation apart from their workspaces: one
 *     operator (gpjc_op) must not be used by two streams at the same time.
 */
#ifndef GPJC_H
#define GPJC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gpjc_status {
  GPJC_OK = 0,
  GPJC_EINVAL = 1,       /* invalid argument or geometry */
  GPJC_ENOMEM = 2,       /* device or host allocation failed */
  GPJC_ECUDA = 3,        /* a CUDA runtime call failed */
  GPJC_ETIMEOUT = 4,     /* a bounded device wait gave up */
  GPJC_ENONFINITE = 5,   /* a non-finite scalar appeared in a reconstruction */
  GPJC_EUNSUPPORTED = 6  /* valid request outside what this build implements */
} gpjc_status;

typedef enum gpjc_precision {
  GPJC_FP32 = 0, /* FP32 data and FFMA compression */
  GPJC_BF16 = 1, /* BF16 operands on tensor cores (tcgen05), FP32 accumulation, per-group scale */
  GPJC_FP16 = 2  /* FP16 operands on tensor cores (tcgen05), FP32 accumulation, per-group scale */
} gpjc_precision;

/* Geometry of one slice or volume.  All arrays are host memory, copied by
 * gpjc_plan_create.  Requirements: nx, ny even; nz == 1 (2D) or even;
 * nx, ny, nz products of 2, 3, 5, 7; ntx = os * nx divisible by w;
 * patch_group[p] in [0, n_groups) for p < ntx / w, every group used;
 * 1 <= keep[g] <= nc * w; lines unique, sorted by (kz, ky), inside the grid. */
typedef struct gpjc_geom {
  int32_t nx, ny, nz, nc, os;
  int32_t w, n_groups;
  const int32_t* patch_group; /* [ntx / w] */
  const int32_t* keep;        /* [n_groups] */
  int32_t n_lines;
  const int32_t* line_ky; /* [n_lines] */
  const int32_t* line_kz; /* [n_lines]; NULL for 2D */
  double cycles, kappa_y, kappa_z; /* wave: cycles per readout, peak-to-peak excursion in lines */
} gpjc_geom;

typedef struct gpjc_plan gpjc_plan;     /* geometry + bookkeeping tables */
typedef struct gpjc_groups gpjc_groups; /* compression matrices A_g      */
typedef struct gpjc_op gpjc_op;         /* E_c operator + workspaces     */

/* ------------------------------------------------------------------ misc -- */
const char* gpjc_strerror(gpjc_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* gpjc_last_error(void);
/* Library version string. */
const char* gpjc_version(void);

/* ------------------------------------------------------------------ plan -- */
/* Validates the geometry and builds the bookkeeping (patch offsets
 * off[p] = sum_{q<p} keep[g(q)], N'_tx, first patch of each group,
 * line map) and the device tables.  Synchronous.  *out is owned by the
 * caller and released with gpjc_plan_destroy. */
gpjc_status gpjc_plan_create(const gpjc_geom* geom, gpjc_plan** out);
void gpjc_plan_destroy(gpjc_plan* plan);
/* Compressed readout length N'_tx (Eq. 15). */
gpjc_status gpjc_plan_ntx_c(const gpjc_plan* plan, int32_t* ntx_c);
/* Aliased sets of the phase-encode mask (Sec. 3.4: the pixel sets that
 * alias together, which decouple the least-squares problem): the connected
 * components of the nonzero pattern of F^H M^T M F (|entry| > 1e-9 of the
 * largest), with F the centred unitary phase-encode DFT and M the sampled
 * lines.  h_set_of_row [ny nz] (raster z, y; may be NULL) receives each
 * row's set, the sets numbered in the order of their first row; *n_sets
 * (may be NULL) their number.  Computed on the host at plan creation. */
gpjc_status gpjc_plan_sets(const gpjc_plan* plan, int32_t* h_set_of_row, int32_t* n_sets);
/* Host copies of the bookkeeping: any pointer may be NULL.
 * h_off [ntx/w], h_ref [n_groups] (first patch of each group),
 * h_line_of [nz*ny] (line index of (kz, ky) or -1). */
gpjc_status gpjc_plan_tables(const gpjc_plan* plan, int32_t* h_off, int32_t* h_ref, int32_t* h_line_of);

/* ------------------------------------------------------------------ groups -- */
typedef struct gpjc_build_params {
  int32_t eig_iters;      /* FP64 subspace iterations (0 = default: 1 after the FP32 phase, else 12) */
  int32_t block;          /* subspace block size b (0 = default: min(N_s, max(2 keep, keep + 16), 96)) */
  int32_t keep_gram;      /* keep P_g (FP64) for gpjc_groups_gram                             */
  int32_t eig_iters_fp32; /* FP32 iterations before the FP64 ones (0 = default 6, -1 = none)  */
} gpjc_build_params;

/* Builds every group's compression matrix from coil maps and a ROI
 * (Sec. 2.4 steps 1-2, Eq. 6-12): ROI compaction (raster order, pixels that
 * no coil sees are dropped), Gram P_g in FP64 from the group's first patch,
 * leading eigenvectors by subspace iteration (FP32 iterations on a rounded
 * copy of P_g, then FP64 iterations on P_g) + FP64 Rayleigh-Ritz,
 * A_g = C_g U_g^H (T (x) I_w).
 *   d_coil  [nc][nz][ny][nx] complex64, device
 *   d_roi   [nz][ny][nx] uint8 (nonzero = inside), device
 *   h_T     [nc][nc] complex64 noise-decorrelation matrix (row-major), host, or NULL for identity
 *   params  may be NULL for defaults
 * Synchronises `stream` once (to reject an empty ROI).  The groups keep
 * their scratch (about G N_s^2 complex128 plus N_C x |grid| complex64) for
 * gpjc_groups_rebuild.  *out is released with gpjc_groups_destroy and must
 * not outlive `plan`. */
gpjc_status gpjc_build_groups(const gpjc_plan* plan, const float* d_coil, const uint8_t* d_roi,
                              const float* h_T, const gpjc_build_params* params, void* stream,
                              gpjc_groups** out);

/* Recomputes the groups of a gpjc_build_groups result from new coil maps
 * and ROI of the same geometry, reusing its scratch: asynchronous on
 * `stream`, allocates nothing, synchronises nothing (usable in stream
 * capture).  An empty ROI yields non-finite A (check with gpjc_groups_info_get). */
gpjc_status gpjc_groups_rebuild(gpjc_groups* groups, const float* d_coil, const uint8_t* d_roi, const float* h_T,
                                void* stream);

/* Groups from given matrices (e.g. a stored result, or an external
 * solver): h_A holds A_g row-major [keep_g][N_s] complex64 for g = 0..G-1,
 * concatenated.  Synchronous. */
gpjc_status gpjc_groups_from_matrices(const gpjc_plan* plan, const float* h_A, gpjc_groups** out);
void gpjc_groups_destroy(gpjc_groups* groups);

typedef struct gpjc_groups_info {
  int64_t roi_pixels;  /* |ROI| used by the Gram                        */
  int32_t block;       /* Ritz values per group (b)                     */
  double max_residual; /* max_g max_{k<keep} ||P u - lambda u|| / lambda_0 */
} gpjc_groups_info;
/* Synchronous (reads the device results of the last build). */
gpjc_status gpjc_groups_info_get(const gpjc_groups* groups, gpjc_groups_info* info);
/* h_A: as gpjc_groups_from_matrices.  h_ritz: [n_groups][block] Ritz values,
 * descending (NULL allowed).  Synchronous. */
gpjc_status gpjc_groups_get(const gpjc_groups* groups, float* h_A, double* h_ritz);
/* Gradient of the smoothed isotropic total variation, the TV term of the
 * regularised reconstruction (Eq. 17; Sec. 3.4 uses a smooth approximation):
 *   TV_eps(x) = sum_{y,x} sqrt(|D_x x|^2 + |D_y x|^2 + eps^2) per z-slice,
 *   d_g = D^H (D x / sqrt(|D x|^2 + eps^2)),
 * forward differences, no difference across the last column / row.
 *   d_x, d_g  [nz][ny][nx] complex64, device, caller-owned; d_g must not
 *             alias d_x
 *   eps       > 0, with eps^2 a normal FP32 number (about 1.1e-19 .. 1.8e19)
 * Asynchronous on `stream`; allocates nothing.  GPJC_EINVAL for null or
 * aliased pointers, a dimension < 1 or an eps outside that range;
 * GPJC_ECUDA if the launch fails. */
gpjc_status gpjc_tv_grad(const float* d_x, int32_t nz, int32_t ny, int32_t nx, double eps, float* d_g,
                         void* stream);

/* Kept dimension per group from the eigenvalue spectrum of P_g (Sec. 2.4,
 * Eq. 8: the spectrum quantifies the compressibility and indicates N_s'):
 * h_keep[g] = the smallest k >= 1 with
 *   sum_{i<k} max(lambda_{g,i}, 0) >= threshold * trace_g,
 * or -1 when the m given values do not reach it.
 *   h_eig    [n_groups][m] leading eigenvalues of each group, descending
 *            (e.g. the Ritz values of gpjc_groups_get, m = block), host
 *   h_trace  [n_groups] trace(P_g), host, or NULL to use the sum of the m
 *            given values (all N_s of them given).  trace(P_g) = |ROI| for
 *            every group (gpjc_groups_info_get roi_pixels): each pixel's
 *            normalised encoding vector (Eq. 11) contributes 1
 *   threshold in (0, 1]
 *   h_keep   [n_groups] int32 output, host
 * Host only (no device work, no allocation).  GPJC_EINVAL for a null
 * pointer, n_groups or m < 1, a threshold outside (0, 1] or a negative /
 * non-finite trace; GPJC_ENONFINITE for a non-finite eigenvalue.  A new
 * plan with these keeps takes the first h_keep[g] rows of each A_g
 * (gpjc_groups_from_matrices): rows are in descending eigenvalue order. */
gpjc_status gpjc_keep_from_energy(const double* h_eig, int32_t n_groups, int32_t m, const double* h_trace,
                                  double threshold, int32_t* h_keep);
/* h_P: [n_groups][N_s][N_s] complex128 Gram matrices (needs keep_gram). */
gpjc_status gpjc_groups_gram(const gpjc_groups* groups, double* h_P);
/* h_pix: [roi_pixels] raster indices of the ROI pixels used. */
gpjc_status gpjc_groups_roi(const gpjc_groups* groups, int32_t* h_pix);

/* ------------------------------------------------------------------ compress -- */
/* S'_{l,p} = A_{g(p)} s_{l,p} for every line and patch (Eq. 13).
 *   d_S  [n_lines][nc][ntx] complex64 raw data, device (16-byte aligned for BF16 / FP16)
 *   d_Sc [n_lines][ntx_c]  complex64 output, device
 * GPJC_FP32 contracts in FP32; GPJC_BF16 / GPJC_FP16 stage patch tiles with
 * TMA and run the group GEMMs on the tensor cores with FP32 accumulation:
 * FP16 rounds each operand once, BF16 carries each operand as a BF16 head
 * and a BF16 remainder (three MMAs per K step, about 16 mantissa bits per
 * product).  They need a periodic group map (patch p in group p mod G, G w
 * dividing ntx; the contiguous map with one patch per group is one), else
 * GPJC_EUNSUPPORTED. */
gpjc_status gpjc_compress(const gpjc_groups* groups, const float* d_S, float* d_Sc, gpjc_precision prec,
                          void* stream);

/* ------------------------------------------------------------------ operator -- */
/* Binds groups and coil maps (d_coil is referenced, not copied: it must stay
 * valid and unchanged while the operator lives) and allocates the
 * workspaces.  nchunk: coil chunks of the readout stage (0 = automatic).
 * prec: GPJC_FP32 applies A_g with FP32 FFMA inside the fused readout
 * kernels; GPJC_BF16 / GPJC_FP16 write the readout spectra (FP32 for BF16,
 * whose GEMM splits them into head + remainder; FP16 for FP16) and apply
 * A_g / A_g^H as tensor-core GEMMs (periodic group maps) when patches are at
 * least 8 samples wide (w >= 8); narrower patches (e.g. per-period groups of
 * w = 2) keep the FP32 readout kernels, whose fused contraction is cheaper
 * there than the tensor-core GEMMs and their spectra round trip through HBM
 * (environment GPJC_TC_READOUT=0 / 1 forces either).  Allocates the
 * gpjc_query workspace; GPJC_ENOMEM (and nothing left allocated) when a
 * device allocation fails.  Synchronous. */
gpjc_status gpjc_op_create(const gpjc_groups* groups, const float* d_coil, gpjc_precision prec, int32_t nchunk,
                           gpjc_op** out);
/* Sizes of an operator before it is created (Eq. 15's N'_tx = sum over
 * patches of the kept dimension of the patch's group, Sec. 2.4): *ntx_c
 * receives N'_tx (the row length of S' and of the hybrid matrix), and
 * *workspace_bytes the device bytes gpjc_op_create(groups, ..., prec,
 * nchunk, ...) would allocate (hybrid matrices, partial images, CG / FISTA
 * vectors, scalars and, for BF16 / FP16 with w >= 8, the spectra buffer).  Either
 * output may be NULL.  Host only, no device work.  GPJC_EINVAL for bad
 * arguments, GPJC_EUNSUPPORTED where gpjc_op_create would refuse the
 * precision. */
gpjc_status gpjc_query(const gpjc_groups* groups, gpjc_precision prec, int32_t nchunk, int32_t* ntx_c,
                       uint64_t* workspace_bytes);
/* Measured FP32 FMA throughput of the current device (no counterpart in the
 * paper): the denominator of the FP32 ALU roofline of the readout kernels.
 * Runs SM count x 8 blocks of 256 threads, eight independent FMA chains of
 * `iters` iterations per thread (after one warm-up launch), times it with
 * CUDA events and writes TFLOP/s (2 flops per FMA) to *tflops.
 * Synchronous; allocates 16 bytes of device memory for its inputs. */
gpjc_status gpjc_probe_fp32_tflops(int32_t iters, double* tflops);
/* Test hook for the out-of-memory paths (no counterpart in the paper): after
 * gpjc_debug_fail_allocations(n) the library's (n+1)-th and later device
 * allocations fail with GPJC_ENOMEM without calling cudaMalloc; n < 0
 * restores normal allocation.  Process-wide. */
void gpjc_debug_fail_allocations(int64_t n);
void gpjc_op_destroy(gpjc_op* op);
/* Nonlinear local-B0 modulation (Sec. 2.1-2.2, Eq. 2-3; the paper's
 * primary hardware case): the modulation phase
 *   phi(t, r) = sum_l a_l(t) B_l(r)
 * of local B0 coils depends on the readout position, so the readout is not
 * a DFT.  The operator stores each phase-encode row's compressed readout
 * encoding matrix (Eq. 14)
 *   G_row[off_p + k][x] = sum_{n,tau} A_{g(p)}[k][n w + tau] c_n(r)
 *                         exp(-i [2 pi t_c x_c / N_tx + phi(p w + tau, r)]) / sqrt(N_tx)
 * ([ny nz][ntx_c][nx] complex64 in device memory, built here on the device)
 * and applies it as a batched matrix-vector product, followed by the
 * phase-encode DFT and line gather of gpjc_apply_E.  The plan's wave
 * parameters are not used by this operator.
 *   d_coil   [nc][nz][ny][nx] complex64, device (referenced, as gpjc_op_create)
 *   d_fields [n_fields][nz][ny][nx] float32 (radians at unit drive), device;
 *            read during this call only
 *   h_amps   [n_fields][ntx] float64 drive a_l(t), host
 * Creates an FP32 operator: gpjc_apply_E / gpjc_apply_EH / gpjc_apply_normal
 * / gpjc_recon (all algorithms) use the stored matrices;
 * gpjc_simulate(_adjoint) return GPJC_EUNSUPPORTED for it, and
 * gpjc_op_autotune keeps its fixed split.  Allocates the gpjc_query
 * workspace plus 8 ny nz ntx_c nx bytes; synchronous.  GPJC_EINVAL for
 * null or non-finite inputs or n_fields outside [0, 64]. */
gpjc_status gpjc_op_create_local_b0(const gpjc_groups* groups, const float* d_coil, int32_t n_fields,
                                    const float* d_fields, const double* h_amps, gpjc_op** out);
/* Times the readout-stage coil-chunk choices on `stream` and keeps the
 * fastest (synchronous): the adjoint's chunk count, then the forward's (each
 * among 1-6, 8, 10, 12, 16, 24, 32 within the workspace's planes, skipping
 * counts that would leave a chunk of coils empty), and
 * for tensor-core readouts (BF16 / FP16, w >= 8) the number of row pieces (1-8)
 * in which the adjoint's tensor-core expansion and inverse readout FFT run
 * (the FP32 spectra of one piece stay in L2; the results do not depend on
 * the split).  *nchunk receives the forward chunk count (may be NULL). */
gpjc_status gpjc_op_autotune(gpjc_op* op, void* stream, int32_t* nchunk);
/* The operator's current launch knobs (set at creation or by
 * gpjc_op_autotune): coil chunks of the forward and of the adjoint readout
 * stage, row pieces of the 16-bit adjoint.  Where the FP32 forward readout
 * runs its balanced one-wave launch (plans whose row blocks make fewer than
 * four waves of the device's resident blocks, e.g. a 256 x 256 slice), the
 * forward chunk count is kept but has no effect (the autotuner skips it).
 * Any output may be NULL. */
gpjc_status gpjc_op_tuning(const gpjc_op* op, int32_t* nchunk, int32_t* nchunk_adj, int32_t* adj_pieces);
/* Sets those knobs (e.g. from a persisted autotuning result): nchunk in
 * [1, the forward workspace's planes], nchunk_adj in [1, the adjoint's],
 * adj_pieces in [1, 8]; results do not depend on them beyond FP32 rounding
 * order.  GPJC_EINVAL outside the ranges, GPJC_EUNSUPPORTED for the
 * stored-matrix operator.  Host only. */
gpjc_status gpjc_op_set_tuning(gpjc_op* op, int32_t nchunk, int32_t nchunk_adj, int32_t adj_pieces);

/* y = E_c x (Eq. 15): d_x [nz][ny][nx] -> d_y [n_lines][ntx_c]. */
gpjc_status gpjc_apply_E(const gpjc_op* op, const float* d_x, float* d_y, void* stream);
/* x = E_c^H y: d_y [n_lines][ntx_c] -> d_x [nz][ny][nx]. */
gpjc_status gpjc_apply_EH(const gpjc_op* op, const float* d_y, float* d_x, void* stream);
/* x_out = E_c^H E_c x_in; if h_or_d_qq is non-NULL (device double) it receives ||E_c x_in||^2. */
gpjc_status gpjc_apply_normal(const gpjc_op* op, const float* d_x, float* d_out, double* d_qq, void* stream);

/* Uncompressed acquisition model (Eq. 4), for simulation and baselines:
 * d_S [n_lines][nc][ntx] = E d_x, and its adjoint. */
gpjc_status gpjc_simulate(const gpjc_op* op, const float* d_x, float* d_S, void* stream);
gpjc_status gpjc_simulate_adjoint(const gpjc_op* op, const float* d_S, float* d_x, void* stream);

/* ------------------------------------------------------------------ recon -- */
/* GPJC_DECOUPLED: the hybrid-space reconstruction (Sec. 3.4, algorithm #1,
 * Eq. 16): the least-squares problem decouples over the aliased sets of
 * the phase-encode mask (gpjc_plan_sets); every set runs its own CG (own
 * alpha, beta, stopping when its ||r||^2 == 0) on its readout subproblem.
 * The history holds the sum over the sets of ||r||^2. */
typedef enum gpjc_alg { GPJC_CG = 0, GPJC_FISTA = 1, GPJC_DECOUPLED = 2 } gpjc_alg;

typedef struct gpjc_recon_params {
  int32_t alg;          /* gpjc_alg                                                  */
  int32_t iters;        /* CG / FISTA iterations (exactly this many)                 */
  double lambda;        /* FISTA: l1 weight on Haar detail coefficients             */
  double lipschitz;     /* FISTA: step 1/L; <= 0 => power iteration from E_c^H S'   */
  int32_t power_iters;  /* power iterations when lipschitz <= 0 (0 = 20)             */
  int32_t haar_levels;  /* FISTA: Haar levels J (nx, ny divisible by 2^J, J <= 5)   */
  int32_t use_x0;       /* nonzero: d_x holds the starting image                     */
  int32_t use_graph;    /* nonzero: capture the iteration loop in a CUDA graph      */
  double lambda_tv;     /* FISTA: weight of the smoothed isotropic TV (Eq. 17), 0 = off */
  double tv_eps;        /* FISTA: TV smoothing eps (> 0, eps^2 a normal FP32 number)     */
} gpjc_recon_params;

typedef struct gpjc_recon_info {
  int32_t status;      /* gpjc_status of the device-side checks                   */
  double lipschitz;    /* L used by FISTA                                          */
  double* h_history;   /* optional host [iters + 1]: CG ||r||^2 per iteration      */
} gpjc_recon_info;

/* Compressed reconstruction of d_Sc [n_lines][ntx_c] into d_x [nz][ny][nx]
 * (Sec. 3.4): CG-SENSE (CGNR on E_c^H E_c x = E_c^H S', Eq. 16's least
 * squares) or FISTA for 1/2 ||E_c x - S'||^2 + lambda ||W x||_1 (orthonormal
 * Haar detail bands) + lambda_tv TV_eps(x) (Eq. 17, TV by its smooth
 * approximation in the gradient step; gpjc_tv_grad's definition).  With
 * lipschitz <= 0 the step size comes from power iteration of E_c^H E_c, plus
 * 8 lambda_tv / tv_eps (the TV gradient's Lipschitz bound); a given
 * lipschitz must bound the whole gradient.  The loop runs on the device
 * without host synchronisation; the call synchronises `stream` once at the
 * end when `info` is non-NULL (to report status, L and history), and then
 * returns GPJC_ENONFINITE when a non-finite step scalar appeared. */
gpjc_status gpjc_recon(const gpjc_op* op, const float* d_Sc, float* d_x, const gpjc_recon_params* params,
                       gpjc_recon_info* info, void* stream);

/* ------------------------------------------------------------------ batch -- */
/* Many 2D slices (each with its own plan, groups and FP32 operator; sizes,
 * coil counts, oversampling and groups may differ) reconstructed by CG in
 * one persistent cooperative launch: every (slice, stage, tile) is a work
 * item of a device queue, and an item waits (bounded) for the previous stage
 * of its slice.  The slices' operators must not be used elsewhere while the
 * batch runs.  Creation allocates the queue and counters (synchronous). */
typedef struct gpjc_batch gpjc_batch;
gpjc_status gpjc_batch_create(int32_t n, gpjc_op* const* ops, int32_t iters, gpjc_batch** out);
void gpjc_batch_destroy(gpjc_batch* batch);
/* CG with x0 = 0 and exactly `iters` iterations per slice (the recurrences
 * of gpjc_recon with alg = GPJC_CG).  d_Sc[i] [n_lines_i][ntx_c_i] in,
 * d_x[i] [ny_i][nx_i] out: host arrays of device pointers.  use_graph: replay
 * a captured graph (memsets + the persistent kernel) while the pointers stay
 * the same.  h_status (may be NULL): device status after a synchronisation. */
gpjc_status gpjc_recon_batched(gpjc_batch* batch, const float* const* d_Sc, float* const* d_x, int32_t use_graph,
                               int32_t* h_status, void* stream);
/* Budget of each dependency wait in SM clock cycles (default 4e9, about 2 s);
 * when a wait runs out the launch aborts and reports GPJC_ETIMEOUT.  Tests
 * set a tiny budget to exercise that path without faulting anything. */
gpjc_status gpjc_batch_set_wait_budget(gpjc_batch* batch, int64_t cycles);
/* Blocks of the persistent launch and work items of one reconstruction. */
gpjc_status gpjc_batch_info(const gpjc_batch* batch, int32_t* grid, int64_t* items);

/* ------------------------------------------------------------------ multi-slice graph -- */
/* Many reconstructions in one CUDA graph (the batched form for slices of
 * uneven size, coil count and precision, 2D or 3D): the slices'
 * reconstructions (gpjc_recon's CG or decoupled CG, same recurrences and
 * results) are captured on n_branches parallel branches and replayed with
 * one graph launch, so one slice's small grids, tails and launch gaps are
 * filled by the others.  Slices go longest first (rows x coils x N_tx) to the
 * least-loaded branch.  Each operator appears once and must not be used
 * elsewhere while the graph runs.  Creation makes the branch streams and
 * events and allocates one status word per slice (synchronous). */
typedef struct gpjc_multi gpjc_multi;
gpjc_status gpjc_multi_create(int32_t n, gpjc_op* const* ops, int32_t n_branches, gpjc_multi** out);
void gpjc_multi_destroy(gpjc_multi* multi);
/* d_Sc[i] [n_lines_i][ntx_c_i] in, d_x[i] image out (x0 = 0), params as
 * gpjc_recon (alg GPJC_CG or GPJC_DECOUPLED, use_x0 / use_graph ignored:
 * always captured; the graph is cached for the same pointers and params, the
 * first call also runs each slice once eagerly).  h_status (may be NULL):
 * the worst device status after a synchronisation of `stream`. */
gpjc_status gpjc_recon_multi(gpjc_multi* multi, const float* const* d_Sc, float* const* d_x,
                             const gpjc_recon_params* params, int32_t* h_status, void* stream);

/* ------------------------------------------------------------------ no allocation -- */
/* x = E_c^H y without any allocation: the paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc on the path
 * where they apply the adjoint -- for example code that runs inside a
 * component that forbids device allocation after start-up (cudaMalloc and
 * cudaFree synchronise the device and can fail under a fixed memory budget),
 * so it cannot create the workspace of a gpjc_op.  It needs only `groups`
 * (and its plan), created once at start-up, and the caller's buffers:
 *   d_coil [nc][nz][ny][nx], d_y [n_lines][ntx_c] in, d_x [nz][ny][nx] out
 *   (complex64, device), with the same layouts and result as gpjc_apply_EH.
 * Scratch: a static 32 MiB device array inside the library, held on every
 * GPU that loads the library until the process exits; geometries whose
 * hybrid matrix (rows x ntx_c complex64, twice that in 3D) exceeds it are
 * rejected with GPJC_EINVAL before any launch, and so are buffers that are
 * not device memory of the current device.  Calls allocate nothing and
 * free nothing.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, and again when
 * the device's context has changed since (after cudaDeviceReset): make that
 * first call before any stream capture.  Every call on a device shares the one
 * array and overwrites all of it that it reads, so no state carries over;
 * calls whose execution overlaps on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller. */
gpjc_status gpjc_apply_EH_static(const gpjc_groups* groups, const float* d_coil, const float* d_y, float* d_x,
                                 void* stream);

/* ------------------------------------------------------------------ profiling -- */
/* Kernels launched by this library in this process (graph replays add the
 * kernel nodes of the replayed graph).  Thread-safe. */
uint64_t gpjc_launch_count(void);

typedef enum gpjc_stage {
  GPJC_STAGE_READOUT_FWD = 0,  /* coil multiply + readout FFT + wave PSF + A_g (E_c, first half) */
  GPJC_STAGE_PHASE_ENCODE = 1, /* phase-encode FFTs, line gather / scatter / mask projection     */
  GPJC_STAGE_READOUT_ADJ = 2   /* A_g^H + inverse readout FFT + conj(coil) sum (E_c^H, second half) */
} gpjc_stage;

/* Enables (1) or disables (0) CUDA-event timing of each operator stage on the
 * stream the stage runs on; enabling clears earlier marks.  Reconstruction
 * calls restart the marks.  Not thread-safe with concurrent use of `op`. */
gpjc_status gpjc_op_profile(gpjc_op* op, int32_t enable);
/* Sum of the device durations of the marked launches of `stage` since the
 * last reset, and their number.  Waits for the marked events. */
gpjc_status gpjc_op_profile_read(const gpjc_op* op, int32_t stage, double* total_ms, int32_t* count);

#ifdef __cplusplus
}
#endif
#endif /* GPJC_H */
