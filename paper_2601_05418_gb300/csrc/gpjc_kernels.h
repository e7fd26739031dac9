// Kernel launchers (host functions defined in the kernel translation units).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "gpjc_internal.h"

namespace gpjc {

// ---- plan tables (k_groups.cu)
cudaError_t launch_make_tables(Geo& g, float2* tw_x, float2* tw_y, float2* tw_z, float2* pre, float* ay,
                               float* az, double cycles, double kappa_y, double kappa_z, cudaStream_t st);
cudaError_t launch_make_post(const Geo& g, float2* post_y, float2* post_z, double cycles, double kappa_y,
                             double kappa_z, cudaStream_t st);

// ---- operator (k_operator.cu)
cudaError_t launch_k1_fwd_fp32(const Geo& g, const float2* x, const float2* coil, const float2* AT,
                               float2* Hpart, int nchunk, cudaStream_t st);
cudaError_t launch_k1_adj_fp32(const Geo& g, const float2* H2, const float2* coil, const float2* A,
                               float2* xpart, int nchunk, cudaStream_t st);
cudaError_t launch_sim_fwd(const Geo& g, const float2* x, const float2* coil, float2* V, int nchunk,
                           cudaStream_t st);
// rows [row0, row0 + nrows) only
cudaError_t launch_sim_fwd_rows(const Geo& g, const float2* x, const float2* coil, float2* V, int nchunk, int row0,
                                int nrows, cudaStream_t st);
cudaError_t launch_sim_adj(const Geo& g, const float2* V, const float2* coil, float2* xpart, int nchunk,
                           cudaStream_t st);
// gradient of the smoothed isotropic TV of each z-slice (k_tv.cu)
cudaError_t launch_tv_grad(const float2* u, float2* g, int nz, int ny, int nx, float eps2, cudaStream_t st);
// rows [row0, row0 + nrows) only (the other rows' partial images are untouched)
cudaError_t launch_sim_adj_rows(const Geo& g, const float2* V, const float2* coil, float2* xpart, int nchunk,
                                int row0, int nrows, cudaStream_t st);
cudaError_t launch_pe_fwd(const Geo& g, const float2* Hpart, int nchunk, int ncols, float2* T, float2* Sc,
                          cudaStream_t st);
cudaError_t launch_pe_adj(const Geo& g, const float2* Sc, int ncols, float2* T, float2* H, cudaStream_t st);
cudaError_t launch_pe_normal(const Geo& g, const float2* Hpart, int nchunk, int ncols, float2* T, float2* H2,
                             double* partials, unsigned* counter, double* qq, cudaStream_t st);
int pe_normal_blocks(const Geo& g, int ncols);

// ---- register-tiled readout stage (k_readout_f.cu, k_readout_a.cu, k_readout_a2.cu)
struct ReadoutGeomHost {
  int G, w, ntx, ntxc;
  std::vector<int> pg, keep, poff, aoff;
};
void build_readout_tiles(const ReadoutGeomHost& h, int rb, bool adjoint, int ts, std::vector<int4>* hdr,
                         std::vector<int4>* cols);
// share of the register tiles' patch columns that hold a column (tiles of 4
// columns over rb rows x the group's patches per row), weighted by the tiles
double readout_col_fill(const ReadoutGeomHost& h, int rb, bool adjoint, int ts);
int readout_tile_count(const ReadoutGeomHost& h, int rb, bool adjoint, int ts);
size_t readout_fwd_smem(const Geo& g, int rb);
size_t readout_adj_smem(const Geo& g, int rb, int hstage);
constexpr int kReadoutMaxNb = 4;  // coils per batched-transform step of k1f_batched
size_t readout_fwd2_smem(const Geo& g, int rb, int nb);
cudaError_t launch_k1f_batched(const Geo& g, const RTiles& tl, const float2* x, const float2* coil,
                               const float2* AT, float2* Hpart, int nchunk, bool balanced, cudaStream_t st);
int k1f_batched_resident(const Geo& g, const RTiles& tl);  // resident blocks on the device (0: unknown)
cudaError_t launch_k1f_tiled(const Geo& g, const RTiles& tl, const float2* x, const float2* coil,
                             const float2* AT, float2* Hpart, int nchunk, cudaStream_t st);
cudaError_t launch_k1a_tiled(const Geo& g, const RTiles& tl, const float2* H2, const float2* coil,
                             const float2* A, float2* xpart, int nchunk, cudaStream_t st);
cudaError_t launch_k1a_tiled_ts2(const Geo& g, const RTiles& tl, const float2* H2, const float2* coil,
                                 const float2* A, float2* xpart, int nchunk, cudaStream_t st);

// ---- batched persistent CG (k_batch.cu)
size_t batch_pe_smem(const Geo& g);
cudaError_t launch_batch_cg(const BatchPlan& bp, int grid, size_t smem, cudaStream_t st);
int batch_max_blocks(size_t smem);

// ---- tensor-core compression (k_tc.cu)
bool make_tc_tmap(const TcGeom& t, const void* base, int lines, int ebytes, CUtensorMap* map);
// fmt 1 = BF16 (head + remainder images, three MMAs per K step; FP32 sources
// only), 0 = FP16 (one image)
size_t tc_compress_smem(const TcGeom& t, int fmt);
size_t tc_expand_smem(const TcGeom& t, int fmt);
size_t tc_pack_comp_elems(const TcGeom& t, int fmt);  // uint16 elements of all compression images
size_t tc_pack_exp_elems(const TcGeom& t, int fmt);   // uint16 elements of all expansion images
cudaError_t launch_tc_pack(const TcGeom& t, int fmt, const float2* A, const float* scale, uint16_t* Bc,
                           uint16_t* Bx, cudaStream_t st);
// lines [line0, lines) (line0 a multiple of the tile's line count)
cudaError_t launch_tc_compress(const CUtensorMap& map, const TcGeom& t, int fmt, int src_bytes, const uint16_t* Bc,
                               float2* out, int line0, int lines, int* status, cudaStream_t st);
cudaError_t launch_tc_expand(const TcGeom& t, int fmt, const float2* H, const uint16_t* Bx, float2* V, int rows,
                             int* status, cudaStream_t st);
size_t tc_gram2_smem(const Geo& g);
cudaError_t launch_tc_gram2(const Geo& g, const float2* chat, const int* pix, const int* dK, int Kpad,
                            const int* pref, const int2* cpairs, int npairs, double2* P, int* status,
                            cudaStream_t st);
cudaError_t launch_sim_fwd_f16(const Geo& g, const float2* x, const float2* coil, void* V, int nchunk,
                               int row0, int nrows, cudaStream_t st);
cudaError_t launch_sim_adj_f16(const Geo& g, const void* V, const float2* coil, float2* xpart, int nchunk,
                               cudaStream_t st);

// ---- groups (k_groups.cu)
cudaError_t launch_roi_count(const Geo& g, const float2* coil, const uint8_t* roi, int* blockcount, int nblk,
                             cudaStream_t st);
cudaError_t launch_roi_scan(const int* blockcount, int* blockoff, int nblk, int* total, cudaStream_t st);
cudaError_t launch_roi_compact(const Geo& g, const float2* coil, const uint8_t* roi, const int* blockoff,
                               int* pix, int nblk, cudaStream_t st);
cudaError_t launch_roi_coils(const Geo& g, const float2* coil, const float2* T, const int* pix, const int* dK,
                             int Kpad, float2* chat, cudaStream_t st);
int roi_block_pixels();
cudaError_t launch_gram(const Geo& g, const float2* chat, const int* pix, const int* dK, int Kpad,
                        const int* pref, double2* P, cudaStream_t st);
cudaError_t launch_hermitize(const Geo& g, double2* P, cudaStream_t st);
cudaError_t launch_eig_init(const Geo& g, int b, double2* X, cudaStream_t st);
cudaError_t launch_eig_matmul(const Geo& g, int b, const double2* P, const double2* X, double2* Y,
                              cudaStream_t st);
cudaError_t launch_eig_orth(const Geo& g, int b, double2* Y, cudaStream_t st);
cudaError_t launch_to_f32(const double2* a, float2* b, size_t n, cudaStream_t st);
cudaError_t launch_to_f64(const float2* a, double2* b, size_t n, cudaStream_t st);
cudaError_t launch_eig_matmul32(const Geo& g, int b, const float2* P, const float2* X, float2* Y, cudaStream_t st);
cudaError_t launch_eig_orth32(const Geo& g, int b, float2* Y, cudaStream_t st);
cudaError_t launch_eig_project(const Geo& g, int b, const double2* Q, const double2* Z, double2* Hm,
                               cudaStream_t st);
cudaError_t launch_eig_jacobi(const Geo& g, int b, double2* Hm, double2* W, double* ritz, int* order,
                              int max_sweeps, cudaStream_t st);
cudaError_t launch_eig_rotate(const Geo& g, int b, const double2* Q, const double2* W, const int* order,
                              double2* U, cudaStream_t st);
cudaError_t launch_eig_residual(const Geo& g, int b, const double2* PU, const double2* U, const double* ritz,
                                const int* order, double* resid, cudaStream_t st);
cudaError_t launch_form_A(const Geo& g, int b, const double2* U, const float2* T, float2* A, float2* AT,
                          float* scale, cudaStream_t st);
cudaError_t launch_compress_fp32(const Geo& g, const float2* S, int n_lines_in, const float2* AT, float2* Sc,
                                 cudaStream_t st);

// ---- nonlinear local-B0 operator: stored compressed readout matrices (k_lb0.cu)
int lb0_build_tile(int ns);  // x tile of the build (0: N_s too large)
cudaError_t launch_lb0_build(const Geo& g, int nfields, const float2* coil, const float* fields, const float* amps,
                             const float2* A, float2* G, cudaStream_t st);
cudaError_t launch_lb0_fwd(const Geo& g, const float2* G, const float2* x, float2* H, cudaStream_t st);
cudaError_t launch_lb0_adj(const Geo& g, const float2* G, const float2* H2, float2* xpart, int nsplit, cudaStream_t st);

// ---- FP32 FMA throughput probe (k_probe.cu): synchronous, on the default stream
cudaError_t probe_fma_tflops(int iters, double* tflops);

// ---- recon (k_recon.cu)
cudaError_t launch_sum_parts(const float2* parts, int nchunk, size_t L, float2* out, double* partials,
                             unsigned* counter, double* nrm2, cudaStream_t st);
int sum_parts_blocks(size_t L);
cudaError_t launch_cg_update1(const float2* parts, int nchunk, size_t L, float2* x, float2* r, const float2* p,
                              const double* rr, const double* qq, double* partials, unsigned* counter,
                              double* rr_new, double* hist, int* status, cudaStream_t st);
cudaError_t launch_cg_update2(float2* p, const float2* r, size_t L, const double* rr, const double* rr_new,
                              cudaStream_t st);
cudaError_t launch_axpby(float2* y, const float2* a, const float2* b, float alpha, float beta, size_t L,
                         cudaStream_t st);
cudaError_t launch_scale_by(float2* v, const float2* src, const double* nrm2, size_t L, double* Lout,
                            cudaStream_t st);
// tvg: smoothed-TV gradient of y (nullptr: no TV term), weighted by lam_tv
cudaError_t launch_fista_step(const Geo& g, const float2* parts, int nchunk, float2* x, float2* y,
                              const float2* b, const double* Lip, double lam, int levels, double ck,
                              const float2* tvg, double lam_tv, int* status, cudaStream_t st);
cudaError_t launch_add_scalar(double* d, double v, cudaStream_t st);
// per-aliased-set CG (hybrid-space reconstruction): one block per image row
cudaError_t launch_ds_rowdot(const float2* parts, int nchunk, size_t L, int rows, int nx, float2* out,
                             const float2* a, double* rowval, cudaStream_t st);
cudaError_t launch_ds_setsum(const double* rowval, const int* ptr, const int* rows, int n_sets, double* out,
                             double* total, cudaStream_t st);
cudaError_t launch_ds_update1(int rows, int nx, const int* set_of_row, float2* x, float2* r, const float2* p,
                              const float2* q, const double* rr, const double* pap, double* rowval, int* status,
                              cudaStream_t st);
cudaError_t launch_ds_update2(int rows, int nx, const int* set_of_row, float2* p, const float2* r, const double* rr,
                              const double* rr_new, cudaStream_t st);
cudaError_t launch_copy(float2* dst, const float2* src, size_t n, cudaStream_t st);
cudaError_t launch_zero(float2* dst, size_t n, cudaStream_t st);
cudaError_t launch_set_scalar(double* d, double v, cudaStream_t st);

}  // namespace gpjc
