// m1_internal.h — host-side launch interface between the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "../../include/m1.h"
#include "m1_device.cuh"

namespace m1 {

constexpr int kMaxRestart = 30;  // GMRES(m) basis bound, m <= 30

// ----------------------------------------------------------------- stencils (m1_stencil.cu)
// time-n face data: lambda+-, alpha on every face of every axis (FP64)
void launch_faces_time_n(const Dev<double>& g, double* const lam_p[3], double* const lam_m[3],
                         double* const alpha[3], cudaStream_t s);
// residual of every cell and, when partials is not null, the partial sums of
// squares (one per block); returns the number of partials written (at most
// capacity: the 2D tiled kernel is used when its tile count fits)
int launch_residual_f64(const Dev<double>& g, const double* U, double* R, double* partials, long long capacity,
                        cudaStream_t s);
// J v from the pressure Jacobian dP/dU frozen at the Newton iterate (2D,
// frozen or fixed wave speeds): launch_pressure_jacobian_f64/_f32 fill dP/dU
// at U (pressure_jacobian_size(g) planes of N, in the precision of the J v
// that applies it), the linear kernels apply it; U (in the kernel's precision)
// serves the ghosts
bool jv_linear_available(const Dev<double>& g);
int pressure_jacobian_size(const Dev<double>& g);
void launch_pressure_jacobian_f64(const Dev<double>& g, const double* U, double* pj, cudaStream_t s);
void launch_pressure_jacobian_f32(const Dev<float>& g, const float* U, float* pj, cudaStream_t s);
void launch_jv_linear_f64(const Dev<double>& g, const double* U, const double* pj, const double* v, double* Jv,
                          cudaStream_t s);
void launch_jv_linear_f32(const Dev<float>& g, const float* U, const float* pj, const float* v, float* Jv,
                          cudaStream_t s);
// Double-word FP64 arithmetic (m1_df.cuh) is allowed for a grid whose scalars c,
// a_r (with gas) and dx lie within 2^-30 .. 2^30: with states and residuals
// below the residual's range guard (2^100) no intermediate then leaves FP32's
// exponent range
inline bool fp64_df_scalars_ok(double c, double a_r, bool gas, int dim, const double* dx) {
    auto ok = [](double x) { return fabs(x) >= 0x1p-30 && fabs(x) <= 0x1p30; };
    if (!ok(c) || (gas && !ok(a_r))) return false;
    for (int a = 0; a < dim; ++a)
        if (!ok(dx[a])) return false;
    return true;
}
// 3D J v tiled in x-y and marching in z (m1_stencil3d.cu): for wave speeds frozen at time n or
// fixed; false (nothing launched) otherwise
bool launch_jv3d_tiled_f64(const Dev<double>& g, const double* U, const double* v, double* Jv, cudaStream_t s);
bool launch_jv3d_tiled_f32(const Dev<float>& g, const float* U, const float* v, float* Jv, cudaStream_t s);
// J M^-1 v with the point-block inverse binv (NU x NU row-major planes, FP32)
// applied to v inside the stencil (M^-1 v is never stored)
void launch_jv_linear_pre_f32(const Dev<float>& g, const float* U, const float* pj, const float* binv,
                              const float* v, float* Jv, cudaStream_t s);
// ----------------------------------------------------------------- BiCGStab (m1_bicgstab.cu)
// device scalars of the recurrence (doubles) and the finish modes
constexpr int kBsRho = 0, kBsAlpha = 1, kBsOmega = 2, kBsBeta = 3, kBsRR = 4, kBsBreak = 5, kBsScalars = 8;
constexpr int kBsModeRho = 0, kBsModeAlpha = 1, kBsModeOmega = 2;
int bs_partial_rows();  // doubles of the partials buffer
// nd (1 or 2) dot products (a0, b0) [, (a1, b1)] summed in a fixed order, then the
// mode's scalar update; kBsModeRho also copies (||r||^2, breakdown) to host_slot if set
void launch_bs_dots_f64(const double* a0, const double* b0, const double* a1, const double* b1, long long n, int nd,
                        double* part, int mode, double* sc, double* host_slot, cudaStream_t s);
void launch_bs_dots_f32(const float* a0, const float* b0, const float* a1, const float* b1, long long n, int nd,
                        double* part, int mode, double* sc, double* host_slot, cudaStream_t s);
void launch_bs_p_f64(double* p, const double* r, const double* v, const double* sc, long long n, cudaStream_t s);
void launch_bs_p_f32(float* p, const float* r, const float* v, const double* sc, long long n, cudaStream_t s);
void launch_bs_s_f64(double* sv, const double* r, const double* v, const double* sc, long long n, cudaStream_t s);
void launch_bs_s_f32(float* sv, const float* r, const float* v, const double* sc, long long n, cudaStream_t s);
// x (FP64) += alpha phat + omega shat; r = s - omega t; then the kBsModeRho finish
void launch_bs_xr_f64(double* x, double* r, const double* phat, const double* shat, const double* sv,
                      const double* t, const double* rhat, double* sc, long long n, double* part, double* host_slot,
                      cudaStream_t s);
void launch_bs_xr_f32(double* x, float* r, const float* phat, const float* shat, const float* sv, const float* t,
                      const float* rhat, double* sc, long long n, double* part, double* host_slot, cudaStream_t s);

// ----------------------------------------------------------------- multigrid (m1_mg.cu)
constexpr int kMgMaxLevels = 16;
// the level-0 operator of the V-cycle: out = J in (FP32, the solver's linear J v)
struct MgJvOp {
    void* ctx;
    void (*apply)(void* ctx, const float* in, float* out, cudaStream_t s);
    // optional fused level-0 passes (with Dinv[0] as M^-1); null: J v plus separate kernels
    void (*down0)(void* ctx, const float* r, float omega, float* z, int nxc, int nyc, float* rc, cudaStream_t s);
    void (*up0)(void* ctx, const float* r, const float* z, const float* zc, int nxc, int nyc, float omega,
                float* zout, cudaStream_t s);
};
// aggregation hierarchy of a 2D grid (FP32): level l is nx[l] x ny[l] cells; A[l]
// the 5-point block stencil (5 n_u^2 planes; A[0] only feeds the coarsening),
// Dinv[l] the inverses of its C blocks (Dinv[0]: the block-Jacobi inverses),
// r/z/z2 per-level work vectors, w0 and probe level-0 work vectors
struct MgHierarchy {
    int nu = 0, nlev = 0;
    bool px = false, py = false;
    int nx[kMgMaxLevels] = {}, ny[kMgMaxLevels] = {};
    float* A[kMgMaxLevels] = {};
    float* Dinv[kMgMaxLevels] = {};
    float* r[kMgMaxLevels] = {};
    float* z[kMgMaxLevels] = {};
    float* z2[kMgMaxLevels] = {};
    float* w0 = nullptr;
    float* probe = nullptr;
};
void mg_plan(MgHierarchy& H, int nu, int nx, int ny, bool px, bool py);
int mg_colour_period(int n, bool periodic);
// direct level-0 assembly from the FP32 descriptor, state and dP/dU (radiation
// only); without it the level-0 stencil is probed through J
struct MgDirect {
    const Dev<float>* g;
    const float* U;
    const float* pj;
};
void mg_build(MgHierarchy& H, const MgJvOp& J, const MgDirect* direct, double* inv64_scratch, int* singular,
              cudaStream_t s);
void mg_cycle(const MgHierarchy& H, const MgJvOp& J, const float* r0, float* zout, cudaStream_t s);
int mg_launches_per_build(const MgHierarchy& H, bool direct);
int mg_launches_per_cycle(const MgHierarchy& H, bool fused);
double mg_cycle_bytes(const MgHierarchy& H, bool fused, bool fixed_eigs);
// level 0 of the multigrid cycle in one tiled pass each (radiation only, FP32):
// down: z = omega M^-1 r, rc = P^T (r - J z); up: zz = z + P zc,
// zout = zz + omega M^-1 (r - J zz); M^-1 the block inverses binv
void launch_mg_down0_f32(const Dev<float>& g, const float* U, const float* pj, const float* binv, const float* r,
                         float omega, float* z, int nxc, int nyc, float* rc, cudaStream_t s);
void launch_mg_up0_f32(const Dev<float>& g, const float* U, const float* pj, const float* binv, const float* r,
                       const float* z, const float* zc, int nxc, int nyc, float omega, float* zout, cudaStream_t s);
// partial-sum entries the residual may need for this grid
long long residual_partial_count(int dim, const int n[3]);
void launch_jv_f64(const Dev<double>& g, const double* U, const double* v, double* Jv, cudaStream_t s);
void launch_jv_f32(const Dev<float>& g, const float* U, const float* v, float* Jv, cudaStream_t s);
void launch_diag_f64(const Dev<double>& g, const double* U, double* blocks, cudaStream_t s);
void launch_block_inverse(int nu, long long N, const double* blocks, double* binv64, float* binv32,
                          int* singular, cudaStream_t s);
// FP32 point blocks (the mixed-precision preconditioner), inverted in FP64
void launch_diag_f32(const Dev<float>& g, const float* U, float* blocks, cudaStream_t s);
void launch_block_inverse_f32(int nu, long long N, const float* blocks, double* binv64, float* binv32,
                              int* singular, cudaStream_t s);
void launch_bj_apply_f64(int nu, long long N, const double* binv, const double* r, double* z, cudaStream_t s);
// block-tridiagonal line preconditioner (1D, FP64): blocks 3 n_u^2 N, factors M and D'^-1 n_u^2 N each
void launch_line_build(const Dev<double>& g, const double* U, double* blocks, double* Mf, double* Dinv,
                       int* singular, cudaStream_t s);
void launch_line_solve(int nu, long long N, const double* blocks, const double* Mf, const double* Dinv,
                       const double* r, double* z, cudaStream_t s);
void launch_bj_apply_f32(int nu, long long N, const float* binv, const float* r, float* z, cudaStream_t s);
// semi-implicit step: hyperbolic update + exchange -> Unew (E, T) and Fstar
void launch_explicit_hyp(const Dev<double>& g, double* Unew, double* Fstar, cudaStream_t s);
// WB source solve along axis b for component b: (I + c dt W_b) F = Fstar
void launch_wb_lines(const Dev<double>& g, int b, const double* Fstar, double* Fout, double* work,
                     cudaStream_t s);
int stencil_blocks(long long N);
// upwind transport of rho c_v T by face velocities u[a] (gas coupling): T* into Tout
// the explicit velocity-dependent radiation sources of the current state into Uout
void launch_velocity_sources(const Dev<double>& g, const double* const u[3], double* Uout, cudaStream_t s);
void launch_advect(const Dev<double>& g, const double* const u[3], double* Tout, cudaStream_t s);

// ----------------------------------------------------------------- Arnoldi (m1_arnoldi.cu)
// device scalars and scratch of one fused Arnoldi step (CGS with selective
// reorthogonalisation, Givens on the FP64 Hessenberg column in the last block)
struct ArnoldiDev {
    long long n, ld;     // vector length, basis stride
    int grid[kMaxRestart];       // blocks of the update pass of Arnoldi step j
    int grid_dots[kMaxRestart];  // blocks of its dots passes (partials holds one row of kMaxRestart + 2 per block)
    double *H, *cs, *sn, *g, *resid, *h1, *h2, *nrm2;
    double* partials;    // one row per block of the first dots pass
    double* partials2;   // and of the second (residual) dots pass
    int* reorth;         // 1 when the second Gram-Schmidt pass runs
    double* resid_host;  // if set: resid[0..2] also written here (mapped pinned host memory)
};
constexpr int kMaxGsBlocks = 4096;  // bound of ArnoldiDev::grid, rows of ArnoldiDev::partials
// blocks of each Arnoldi step's passes for vectors of length n (occupancy of this device)
void arnoldi_grid_table(long long n, bool fp32, int* grid, int* grid_dots);
void launch_arnoldi_step_f64(const ArnoldiDev& K, double* V, double* w, int j, cudaStream_t s);
void launch_arnoldi_step_f32(const ArnoldiDev& K, float* V, float* w, int j, cudaStream_t s);

// ----------------------------------------------------------------- vectors (m1_vec.cu)
int reduce_blocks();
// partial sums of squares of x (FP64) and the final sum into out[0]
void launch_norm2_f64(const double* x, long long n, double* partials, double* out, cudaStream_t s);
void launch_norm2_f32(const float* x, long long n, double* partials, double* out, cudaStream_t s);
void launch_finish_sum(const double* partials, int nparts, int ncols, double* out, cudaStream_t s);
// y = x * (1 / sqrt(*nrm2)), zero when the norm is zero
void launch_scale_inv_sqrt_f64(const double* x, const double* nrm2, double* y, long long n, cudaStream_t s);
void launch_scale_inv_sqrt_f32(const float* x, const double* nrm2, float* y, long long n, cudaStream_t s);
// x += sum_{i<k} y[i] Z_i
void launch_lincomb_add_f64(const double* Z, long long ld, int k, const double* y, double* x, long long n,
                            cudaStream_t s);
void launch_lincomb_add_f32_to_f64(const float* Z, long long ld, int k, const double* y, double* x, long long n,
                                   cudaStream_t s);
void launch_axpy_f64(double a, const double* x, double* y, long long n, cudaStream_t s);  // y += a x
void launch_axpby_f64(double a, const double* x, double b, const double* y, double* out, long long n,
                      cudaStream_t s);  // out = a x + b y
void launch_axpby_f32(float a, const float* x, float b, const float* y, float* out, long long n,
                      cudaStream_t s);  // out = a x + b y (FP32)
void launch_f64_to_f32(const double* x, float* y, long long n, cudaStream_t s);
void launch_f32_to_f64(const float* x, double* y, long long n, cudaStream_t s);
void launch_scale_f64_to_f32(const double* x, const double* nrm2, float* y, long long n, cudaStream_t s);
// back substitution y = H^-1 g on the rotated k x k triangle
void launch_backsolve(const double* H, const double* g, int k, double* y, cudaStream_t s);
// count cells with |F| > c E and non-finite entries
// ----------------------------------------------------------------- admissibility fallback (m1_fallback.cu)
// faces of flagged cells: lambda+- = +-c, alpha = 1 (the FP64 time-n face arrays)
void launch_fallback_faces(const Dev<double>& g, const unsigned char* fb, double* const lam_p[3],
                           double* const lam_m[3], double* const alpha[3], cudaStream_t s);
// flag unflagged cells by rule 0 (E <= 0 or |F| > cE in U; their U is reset to U^n) or rule 1
// (max_k |R_k| >= thresh; U kept), count += cells flagged
void launch_fallback_flag(int rule, int nu, int dim, long long N, double c, double thresh, double* U,
                          const double* R, const double* Un, unsigned char* fb, unsigned long long* count,
                          cudaStream_t s);
// *out = bit pattern of max |R| over all n_u N entries (atomicMax on a zeroed word)
void launch_residual_absmax(int nu, long long N, const double* R, unsigned long long* out, cudaStream_t s);
// per flagged cell: delta *= theta_i so that U + delta stays admissible
void launch_admissible_theta(int nu, int dim, long long N, double c, const double* U, double* delta,
                             const unsigned char* fb, cudaStream_t s);
void launch_realizability(const double* U, int dim, long long N, double c, unsigned long long* count,
                          cudaStream_t s);

// ----------------------------------------------------------------- learned preconditioner (m1_unet.cu)
// z += scale (N([v / scale, stat]) - y0): stat = the four planes of k_nn_static at the Newton
// iterate, y0 = nn_null_response at the same iterate (zero3: 3N zero floats)
m1_status nn_apply_add(m1_nn* nn, const float* v, long long N, const float* stat, const float* y0, float scale,
                       float* z, cudaStream_t s);
// the same with scale = the RMS of v (3N entries) from its squared norm n2[0] on the device
m1_status nn_apply_add_rms(m1_nn* nn, const float* v, long long N, const float* stat, const float* y0,
                           const double* n2, float* z, cudaStream_t s);
m1_status nn_null_response(m1_nn* nn, const float* zero3, long long N, const float* stat, float* y0, cudaStream_t s);
int nn_height(const m1_nn* nn);
int nn_width(const m1_nn* nn);
void launch_logsig(const double* sig, long long N, double dx, float* out, cudaStream_t s);
// the network's opacity and state planes (logsig, f_x, f_y, normalised log E) from U
void launch_nn_static_f64(const double* U, long long N, double c, const float* logsig, float* stat, cudaStream_t s);
void launch_nn_static_f32(const float* U, long long N, double c, const float* logsig, float* stat, cudaStream_t s);
void launch_pack_pair(const double* r, const double* tt, long long N, const float* stat, double scale, float* x,
                      float* t, cudaStream_t s);

}  // namespace m1
