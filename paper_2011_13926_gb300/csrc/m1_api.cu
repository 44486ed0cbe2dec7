// m1_api.cu — the C ABI (include/m1.h): context, data movement, the
// semi-implicit step, and the Newton-Raphson / restarted GMRES driver of the
// backward-Euler step (Sects. 3.3.1-3.3.2 of Bloch et al. 2021).
//
// The host only sequences kernels and reads back scalars (norms, the GMRES
// residual estimate); every vector operation runs on the GPU.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/m1.h"
#include "m1_internal.h"

using namespace m1;

namespace {

constexpr int kHLd = kMaxRestart + 1;   // Hessenberg leading dimension
constexpr int kPartCols = kMaxRestart + 1;

struct Faces64 {
    double* lam_p[3] = {nullptr, nullptr, nullptr};
    double* lam_m[3] = {nullptr, nullptr, nullptr};
    double* alpha[3] = {nullptr, nullptr, nullptr};
};
struct Faces32 {
    float* lam_p[3] = {nullptr, nullptr, nullptr};
    float* lam_m[3] = {nullptr, nullptr, nullptr};
    float* alpha[3] = {nullptr, nullptr, nullptr};
};

// device scalars of one Krylov solve
struct Scal {
    double* nrm2;     // [4]
    double* h1;       // [kPartCols]
    double* h2;       // [kPartCols]
    double* H;        // [kHLd * kMaxRestart]
    double* cs;       // [kMaxRestart]
    double* sn;       // [kMaxRestart]
    double* g;        // [kPartCols]
    double* y;        // [kPartCols]
    double* resid;    // [2]
};

}  // namespace

struct m1_ctx {
    m1_grid_desc d{};
    cudaStream_t s = nullptr;
    int dim = 1, nu = 2;
    long long N = 0, n = 0;
    long long ld = 0;  // Krylov basis stride: n rounded up to 64 elements (256-byte rows)
    long long nfaces[3] = {0, 0, 0};
    long long bM[3] = {0, 0, 0};
    // FP64 fields
    double *sig_a = nullptr, *sig_f = nullptr, *B = nullptr, *S = nullptr, *rho_cv = nullptr;
    double *Un = nullptr, *Unew = nullptr;
    double *bE[3][2] = {}, *bF[3][2] = {};
    unsigned char* bmask[3][2] = {};
    Faces64 f64;
    // FP32 copies for the inner solver
    float *sig_a32 = nullptr, *sig_f32 = nullptr, *B32 = nullptr, *S32 = nullptr, *rho_cv32 = nullptr;
    float* Un32 = nullptr;
    float *bE32[3][2] = {}, *bF32[3][2] = {};
    Faces32 f32;
    bool has_state = false, has_opacity = false, dirty = true, sigf_is_siga = true;
    // work buffers (allocated on first use)
    bool work_ok = false, work32_ok = false, expl_ok = false;
    double *U = nullptr, *R = nullptr, *Ut = nullptr, *Rt = nullptr, *delta = nullptr, *rhs = nullptr;
    double *w = nullptr, *z = nullptr, *tmp = nullptr, *V = nullptr, *xacc = nullptr;
    double *blocks = nullptr, *binv = nullptr;
    float *binv32 = nullptr, *V32 = nullptr, *w32 = nullptr, *z32 = nullptr, *U32 = nullptr, *tmp32 = nullptr;
    double *Fstar = nullptr, *linework = nullptr;
    m1_nn* nn = nullptr;        // learned preconditioner (not owned)
    float* logsig = nullptr;    // its opacity channel
    float* nn_static = nullptr; // its four input planes that are fixed within a linear solve (k_nn_static)
    float* nn_null = nullptr;   // its output for a zero residual at the same iterate (3N, subtracted)
    float* Z32 = nullptr;       // flexible-GMRES basis of preconditioned vectors
    int nn_form = 0;            // how the correction combines with point-block Jacobi (m1_set_learned_form)
    float *nn_r = nullptr, *nn_t = nullptr;  // two-stage form: the residual of the first stage, M^-1 of it
    double *nn_part = nullptr, *nn_n2 = nullptr;  // its squared norm: partial sums and the total
    double* pj64 = nullptr;     // dP/dU at the Newton iterate (2D frozen wave speeds), FP64
    float* pj32 = nullptr;      // the same in FP32
    // multigrid preconditioner (allocated on first use)
    MgHierarchy mg;
    bool mg_alloc = false;
    double* mg_inv64 = nullptr;  // FP64 scratch of the block inverses of every level
    double *line_B = nullptr, *line_M = nullptr, *line_Dinv = nullptr;  // line preconditioner (1D)
    double* bs_part = nullptr;   // BiCGStab: dot-product partials
    double* bs_sc = nullptr;     // BiCGStab: recurrence scalars
    Dev<float> mg_g32{};         // the step's FP32 descriptor the level-0 J v uses
    bool mg_probe = false;       // level-0 stencil by probes through J v instead of directly
    float *pair_x = nullptr, *pair_t = nullptr;  // staging of one training pair (4N and 3N floats)
    double* vel[3] = {nullptr, nullptr, nullptr};  // prescribed face velocities (gas advection)
    double* partials = nullptr;
    double* ar_partials = nullptr;
    int* ar_reorth = nullptr;
    int gs_grid32[kMaxRestart] = {}, gs_grid64[kMaxRestart] = {};  // Gram-Schmidt grids per Arnoldi step
    int gs_dots32[kMaxRestart] = {}, gs_dots64[kMaxRestart] = {};
    long long residual_partials = 0;                                 // entries of partials
    Scal sc{};
    double* scal_base = nullptr;
    int* singular = nullptr;
    unsigned long long* viol = nullptr;
    unsigned char* fb = nullptr;          // admissibility fallback: flagged cells of the current step
    unsigned long long* fbw = nullptr;    // [0] cells flagged by a check, [1] bit pattern of max |R|
    bool fb_on = false;                   // some cell is flagged: the kernels read fb
    long long fb_cells = 0;
    double* hpin = nullptr;      // pinned host scalars (mapped)
    double* hpin_dev = nullptr;  // their device address, or null when mapping is unavailable
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_res[2] = {nullptr, nullptr};  // residual estimate of Arnoldi steps j (even, odd) on the host
    // FP64 arithmetic of the residual and J v stencils (m1_set_fp64_arithmetic):
    // the requested mode, the one in use, and how often the double-word
    // residual's range guard sent a residual back to FP64
    int fp64_mode = M1_FP64_AUTO;
    bool fp64_df_ok = false;  // double words allowed: the mode, the grid's scalars, no range fallback yet
    bool fp64_df = false;     // in use now (M1_FP64_AUTO: decided per implicit step)
    long long fp64_df_fallbacks = 0;
    // per-kernel-class timers (m1_profile)
    bool prof = false;
    std::vector<cudaEvent_t> evs;
    std::vector<int> ev_cls;
    int ev_used = 0;
    m1_stats_t st{};
    std::string err = "no error";
};

namespace {

m1_status fail(m1_ctx* c, m1_status code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? M1_ERR_NOMEM : M1_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

#define CKS(expr)                          \
    do {                                   \
        m1_status st_ = (expr);            \
        if (st_ != M1_OK) return st_;      \
    } while (0)

template <class T>
m1_status dalloc(m1_ctx* ctx, T** p, size_t count) {
    if (*p) return M1_OK;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, M1_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return M1_OK;
}

m1_status copy_in(m1_ctx* ctx, void* dst, const void* src, size_t bytes, m1_mem mem) {
    CK(cudaMemcpyAsync(dst, src, bytes, mem == M1_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->s));
    return M1_OK;
}
m1_status copy_out(m1_ctx* ctx, void* dst, const void* src, size_t bytes, m1_mem mem) {
    CK(cudaMemcpyAsync(dst, src, bytes, mem == M1_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->s));
    return M1_OK;
}
// fold the recorded event pairs into the per-class totals (stream must be idle)
void resolve_timers(m1_ctx* ctx) {
    for (int i = 0; i < ctx->ev_used / 2; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->evs[2 * i], ctx->evs[2 * i + 1]) == cudaSuccess) {
            ctx->st.kernel_ms[ctx->ev_cls[i]] += ms;
            ctx->st.kernel_count[ctx->ev_cls[i]] += 1;
        }
    }
    ctx->ev_used = 0;
}

m1_status sync(m1_ctx* ctx) {
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->s));
    if (ctx->prof) resolve_timers(ctx);
    return M1_OK;
}

// Scoped timer of one kernel class: event records around the enclosed launches.
struct TK {
    m1_ctx* c;
    int slot = -1;
    TK(m1_ctx* ctx, int cls) : c(ctx) {
        if (!c->prof) return;
        if (c->ev_used + 2 > (int)c->evs.size()) {
            cudaStreamSynchronize(c->s);
            resolve_timers(c);
        }
        slot = c->ev_used;
        c->ev_used += 2;
        c->ev_cls[slot / 2] = cls;
        cudaEventRecord(c->evs[slot], c->s);
    }
    ~TK() {
        if (slot >= 0) cudaEventRecord(c->evs[slot + 1], c->s);
    }
};

void count(m1_ctx* ctx, int k) { ctx->st.kernel_launches += k; }

// J v by dual numbers: the 3D tiled kernel where it applies, else the generic path
void jv_f64(const Dev<double>& g, const double* U, const double* v, double* Jv, cudaStream_t s) {
    if (!launch_jv3d_tiled_f64(g, U, v, Jv, s)) launch_jv_f64(g, U, v, Jv, s);
}
void jv_f32(const Dev<float>& g, const float* U, const float* v, float* Jv, cudaStream_t s) {
    if (!launch_jv3d_tiled_f32(g, U, v, Jv, s)) launch_jv_f32(g, U, v, Jv, s);
}

template <class R>
void fill_dev_common(const m1_ctx* ctx, Dev<R>& g) {
    g.dim = ctx->dim;
    g.nx = ctx->d.n[0];
    g.ny = ctx->d.n[1];
    g.nz = ctx->d.n[2];
    g.N = ctx->N;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = ctx->d.n[a];
        const double dx = (ctx->d.hi[a] - ctx->d.lo[a]) / ctx->d.n[a];
        g.dx[a] = (R)dx;
        g.inv_dx[a] = (R)(1.0 / dx);
        g.bM[a] = ctx->bM[a];
        for (int sd = 0; sd < 2; ++sd) g.bc[a][sd] = ctx->d.bc[a][sd];
    }
    g.stride[0] = 1;
    g.stride[1] = ctx->d.n[0];
    g.stride[2] = (long long)ctx->d.n[0] * ctx->d.n[1];
    g.c = (R)ctx->d.c;
    g.a_r = (R)ctx->d.a_r;
    g.lambda_floor = (R)ctx->d.lambda_floor;
    g.gas = ctx->d.gas_coupling;
    g.wb = ctx->d.well_balanced;
    g.ap = ctx->d.ap_correction;
    g.fixed_eigs = ctx->d.fixed_eigs;
    g.wb_boundary = ctx->d.wb_boundary;
    g.implicit_eigs = ctx->d.implicit_eigs;
    g.fb = ctx->fb_on ? ctx->fb : nullptr;
}

Dev<double> dev64(const m1_ctx* ctx, double dt) {
    Dev<double> g{};
    fill_dev_common(ctx, g);
    g.dt = dt;
    g.df = ctx->fp64_df ? 1 : 0;
    g.sig_a = ctx->sig_a;
    g.sig_f = ctx->sig_f;
    g.B = ctx->d.gas_coupling ? nullptr : ctx->B;
    g.S = ctx->S;
    g.rho_cv = ctx->rho_cv;
    g.Un = ctx->Un;
    for (int a = 0; a < 3; ++a) {
        g.alpha[a] = ctx->f64.alpha[a];
        g.lam_p[a] = ctx->f64.lam_p[a];
        g.lam_m[a] = ctx->f64.lam_m[a];
        for (int sd = 0; sd < 2; ++sd) {
            g.bE[a][sd] = ctx->bE[a][sd];
            g.bF[a][sd] = ctx->bF[a][sd];
            g.bmask[a][sd] = ctx->bmask[a][sd];
        }
    }
    return g;
}

Dev<float> dev32(const m1_ctx* ctx, double dt) {
    Dev<float> g{};
    fill_dev_common(ctx, g);
    g.dt = (float)dt;
    g.sig_a = ctx->sig_a32;
    g.sig_f = ctx->sig_f32;
    g.B = ctx->d.gas_coupling ? nullptr : ctx->B32;
    g.S = ctx->S ? ctx->S32 : nullptr;
    g.rho_cv = ctx->rho_cv32;
    g.Un = ctx->Un32;
    for (int a = 0; a < 3; ++a) {
        g.alpha[a] = ctx->f32.alpha[a];
        g.lam_p[a] = ctx->f32.lam_p[a];
        g.lam_m[a] = ctx->f32.lam_m[a];
        for (int sd = 0; sd < 2; ++sd) {
            g.bE[a][sd] = ctx->bE32[a][sd];
            g.bF[a][sd] = ctx->bF32[a][sd];
            g.bmask[a][sd] = ctx->bmask[a][sd];
        }
    }
    return g;
}

m1_status refresh(m1_ctx* ctx);

// validate the inputs; recompute the time-n face data and the FP32 copies
// after any input changed
m1_status prepare(m1_ctx* ctx) {
    if (!ctx->has_state) return fail(ctx, M1_ERR_STATE, "no state: call m1_set_state first");
    if (!ctx->has_opacity) return fail(ctx, M1_ERR_STATE, "no opacity: call m1_set_opacity first");
    for (int a = 0; a < ctx->dim; ++a)
        for (int sd = 0; sd < 2; ++sd)
            if (ctx->d.bc[a][sd] == M1_BC_DIRICHLET && !ctx->bE[a][sd])
                return fail(ctx, M1_ERR_STATE, "Dirichlet boundary without data: call m1_set_boundary");
    if (!ctx->dirty) return M1_OK;
    return refresh(ctx);
}

// time-n face data (lambda+-, alpha) and the FP32 copies of every input
m1_status refresh(m1_ctx* ctx) {
    Dev<double> g = dev64(ctx, 0.0);
    {
    TK t(ctx, M1_K_VECTOR);
    launch_faces_time_n(g, ctx->f64.lam_p, ctx->f64.lam_m, ctx->f64.alpha, ctx->s);
    count(ctx, ctx->dim);
    const long long N = ctx->N;
    launch_f64_to_f32(ctx->sig_a, ctx->sig_a32, N, ctx->s);
    launch_f64_to_f32(ctx->sig_f, ctx->sig_f32, N, ctx->s);
    if (ctx->B) launch_f64_to_f32(ctx->B, ctx->B32, N, ctx->s);
    if (ctx->S) launch_f64_to_f32(ctx->S, ctx->S32, N, ctx->s);
    if (ctx->rho_cv) launch_f64_to_f32(ctx->rho_cv, ctx->rho_cv32, N, ctx->s);
    launch_f64_to_f32(ctx->Un, ctx->Un32, ctx->n, ctx->s);
    for (int a = 0; a < ctx->dim; ++a) {
        launch_f64_to_f32(ctx->f64.alpha[a], ctx->f32.alpha[a], ctx->nfaces[a], ctx->s);
        launch_f64_to_f32(ctx->f64.lam_p[a], ctx->f32.lam_p[a], ctx->nfaces[a], ctx->s);
        launch_f64_to_f32(ctx->f64.lam_m[a], ctx->f32.lam_m[a], ctx->nfaces[a], ctx->s);
        for (int sd = 0; sd < 2; ++sd)
            if (ctx->bE[a][sd]) {
                launch_f64_to_f32(ctx->bE[a][sd], ctx->bE32[a][sd], ctx->bM[a], ctx->s);
                launch_f64_to_f32(ctx->bF[a][sd], ctx->bF32[a][sd], ctx->bM[a] * ctx->dim, ctx->s);
            }
    }
    if (ctx->nn && ctx->logsig)
        launch_logsig(ctx->sig_f, N, (ctx->d.hi[0] - ctx->d.lo[0]) / ctx->d.n[0], ctx->logsig, ctx->s);
    }
    ctx->dirty = false;
    return sync(ctx);
}

m1_status ensure_work(m1_ctx* ctx) {
    if (ctx->work_ok) return M1_OK;
    const long long n = ctx->n, N = ctx->N;
    const int nu = ctx->nu;
    CKS(dalloc(ctx, &ctx->U, n));
    CKS(dalloc(ctx, &ctx->R, n));
    CKS(dalloc(ctx, &ctx->Ut, n));
    CKS(dalloc(ctx, &ctx->Rt, n));
    CKS(dalloc(ctx, &ctx->delta, n));
    CKS(dalloc(ctx, &ctx->rhs, n));
    CKS(dalloc(ctx, &ctx->w, n));
    CKS(dalloc(ctx, &ctx->z, n));
    CKS(dalloc(ctx, &ctx->tmp, n));
    CKS(dalloc(ctx, &ctx->xacc, n));
    CKS(dalloc(ctx, &ctx->V, (size_t)ctx->ld * (kMaxRestart + 1)));
    CKS(dalloc(ctx, &ctx->blocks, (size_t)nu * nu * N));
    CKS(dalloc(ctx, &ctx->binv, (size_t)nu * nu * N));
    CKS(dalloc(ctx, &ctx->binv32, (size_t)nu * nu * N));
    CKS(dalloc(ctx, &ctx->fb, (size_t)N));
    CKS(dalloc(ctx, &ctx->fbw, 2));
    CK(cudaMemsetAsync(ctx->fb, 0, (size_t)N, ctx->s));
    ctx->work_ok = true;
    return M1_OK;
}

m1_status ensure_work32(m1_ctx* ctx) {
    if (ctx->work32_ok) return M1_OK;
    const long long n = ctx->n;
    CKS(dalloc(ctx, &ctx->V32, (size_t)ctx->ld * (kMaxRestart + 1)));
    CKS(dalloc(ctx, &ctx->w32, n));
    CKS(dalloc(ctx, &ctx->z32, n));
    CKS(dalloc(ctx, &ctx->U32, n));
    CKS(dalloc(ctx, &ctx->tmp32, n));
    ctx->work32_ok = true;
    return M1_OK;
}

// ||x||_2 read back to the host (FP64 accumulation)
m1_status norm_f64(m1_ctx* ctx, const double* x, double* out) {
    {
        TK t(ctx, M1_K_ORTHO);
        launch_norm2_f64(x, ctx->n, ctx->partials, ctx->sc.nrm2, ctx->s);
    }
    count(ctx, 2);
    CK(cudaMemcpyAsync(ctx->hpin, ctx->sc.nrm2, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CKS(sync(ctx));
    *out = sqrt(ctx->hpin[0]);
    return M1_OK;
}

// R = R(U) and its norm
m1_status residual_norm(m1_ctx* ctx, const Dev<double>& g0, const double* U, double* R, double* nrm) {
    Dev<double> g = g0;
    g.df = g0.df && ctx->fp64_df_ok;  // a descriptor made before a range fallback
    for (;;) {
        {
            TK t(ctx, M1_K_RESIDUAL);
            const int nb = launch_residual_f64(g, U, R, ctx->partials, ctx->residual_partials, ctx->s);
            launch_finish_sum(ctx->partials, nb, 1, ctx->sc.nrm2, ctx->s);
        }
        count(ctx, 2);
        ctx->st.residual_calls++;
        CK(cudaMemcpyAsync(ctx->hpin, ctx->sc.nrm2, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
        CKS(sync(ctx));
        if (g.df && !std::isfinite(ctx->hpin[0])) {
            // out of the double-word range (or not finite at all): FP64 from here on
            ctx->fp64_df = false;
            ctx->fp64_df_ok = false;
            ctx->fp64_df_fallbacks++;
            g.df = 0;
            continue;
        }
        *nrm = sqrt(ctx->hpin[0]);
        return M1_OK;
    }
}

// M1_FP64_AUTO: the double-word arithmetic when the grid's scalars (c, a_r,
// dx) lie within 2^-30 .. 2^30, so that with states and residuals below the
// range guard's 2^100 no intermediate leaves FP32's exponent range
bool fp64_auto_df(const m1_grid_desc& d) {
    double dx[3];
    for (int a = 0; a < 3; ++a) dx[a] = (d.hi[a] - d.lo[a]) / d.n[a];
    return fp64_df_scalars_ok(d.c, d.a_r, d.gas_coupling != 0, d.dim, dx);
}

// dP/dU at U for the linear J v (2D, frozen or fixed wave speeds); false
// when J v stays on dual numbers
// dP/dU for the linear J v (2D, frozen or fixed wave speeds), in FP64 at U or
// in FP32 at U32 (the FP32 inner solver's own operator); false when J v stays
// on dual numbers
m1_status pressure_jacobian64(m1_ctx* ctx, const Dev<double>& g, const double* U, bool* made) {
    *made = false;
    if (!jv_linear_available(g)) return M1_OK;
    CKS(dalloc(ctx, &ctx->pj64, (size_t)pressure_jacobian_size(g) * ctx->N));
    TK t(ctx, M1_K_PC_BUILD);
    launch_pressure_jacobian_f64(g, U, ctx->pj64, ctx->s);
    count(ctx, 1);
    *made = true;
    return M1_OK;
}
m1_status pressure_jacobian32(m1_ctx* ctx, const Dev<double>& g, const Dev<float>& g32, const float* U32, bool* made) {
    *made = false;
    if (!jv_linear_available(g)) return M1_OK;
    CKS(dalloc(ctx, &ctx->pj32, (size_t)pressure_jacobian_size(g) * ctx->N));
    TK t(ctx, M1_K_PC_BUILD);
    launch_pressure_jacobian_f32(g32, U32, ctx->pj32, ctx->s);
    count(ctx, 1);
    *made = true;
    return M1_OK;
}

// ---------------------------------------------------------------- multigrid
bool mg_supported(const m1_ctx* ctx, const Dev<double>& g) {
    if (!jv_linear_available(g) || ctx->dim != 2) return false;
    for (int a = 0; a < 2; ++a) {
        if (ctx->d.bc[a][0] == M1_BC_PERIODIC && ctx->d.n[a] < 3) return false;
        // the level cap keeps the coarsest level within one CTA (<= 16 cells a side)
        if ((long long)ctx->d.n[a] > (16LL << (kMgMaxLevels - 1))) return false;
    }
    return true;
}

void mg_jv_apply(void* c, const float* in, float* out, cudaStream_t s) {
    m1_ctx* ctx = static_cast<m1_ctx*>(c);
    launch_jv_linear_f32(ctx->mg_g32, ctx->U32, ctx->pj32, in, out, s);
}
void mg_down0(void* c, const float* r, float omega, float* z, int nxc, int nyc, float* rc, cudaStream_t s) {
    m1_ctx* ctx = static_cast<m1_ctx*>(c);
    launch_mg_down0_f32(ctx->mg_g32, ctx->U32, ctx->pj32, ctx->binv32, r, omega, z, nxc, nyc, rc, s);
}
void mg_up0(void* c, const float* r, const float* z, const float* zc, int nxc, int nyc, float omega, float* zout,
            cudaStream_t s) {
    m1_ctx* ctx = static_cast<m1_ctx*>(c);
    launch_mg_up0_f32(ctx->mg_g32, ctx->U32, ctx->pj32, ctx->binv32, r, z, zc, nxc, nyc, omega, zout, s);
}
// the level-0 operator of the cycle: fused passes for radiation only
MgJvOp mg_op(m1_ctx* ctx) {
    const bool fused = ctx->nu == 3;
    return MgJvOp{ctx, mg_jv_apply, fused ? mg_down0 : nullptr, fused ? mg_up0 : nullptr};
}

m1_status ensure_mg(m1_ctx* ctx) {
    if (ctx->mg_alloc) return M1_OK;
    MgHierarchy& H = ctx->mg;
    mg_plan(H, ctx->nu, ctx->d.n[0], ctx->d.n[1], ctx->d.bc[0][0] == M1_BC_PERIODIC,
            ctx->d.bc[1][0] == M1_BC_PERIODIC);
    const size_t nu = (size_t)ctx->nu;
    for (int l = 0; l < H.nlev; ++l) {
        const size_t N = (size_t)H.nx[l] * H.ny[l];
        CKS(dalloc(ctx, &H.A[l], 5 * nu * nu * N));
        if (l > 0) {
            CKS(dalloc(ctx, &H.Dinv[l], nu * nu * N));
            CKS(dalloc(ctx, &H.r[l], nu * N));
        }
        CKS(dalloc(ctx, &H.z[l], nu * N));
        CKS(dalloc(ctx, &H.z2[l], nu * N));
    }
    CKS(dalloc(ctx, &H.w0, nu * ctx->N));
    CKS(dalloc(ctx, &H.probe, nu * ctx->N));
    CKS(dalloc(ctx, &ctx->mg_inv64, nu * nu * (size_t)ctx->N));  // FP64 scratch of the block inverses
    ctx->mg_alloc = true;
    return M1_OK;
}

// the hierarchy at the FP32 state U32 (pj32 and binv32 already built for it)
m1_status build_mg(m1_ctx* ctx, const Dev<float>& g32) {
    CKS(ensure_mg(ctx));
    TK t(ctx, M1_K_PC_BUILD);
    ctx->mg_g32 = g32;
    ctx->mg.Dinv[0] = ctx->binv32;  // written by the build from the level-0 C blocks
    CK(cudaMemsetAsync(ctx->singular, 0, sizeof(int), ctx->s));
    const MgJvOp op = mg_op(ctx);
    const MgDirect direct{&ctx->mg_g32, ctx->U32, ctx->pj32};
    const bool use_direct = ctx->nu == 3 && !ctx->mg_probe;
    mg_build(ctx->mg, op, use_direct ? &direct : nullptr, ctx->mg_inv64, ctx->singular, ctx->s);
    count(ctx, mg_launches_per_build(ctx->mg, use_direct));
    ctx->st.bytes_per_mg_cycle = mg_cycle_bytes(ctx->mg, op.down0 != nullptr, ctx->d.fixed_eigs != 0);
    return M1_OK;
}

void mg_apply(m1_ctx* ctx, const float* in, float* out) {
    const MgJvOp op = mg_op(ctx);
    mg_cycle(ctx->mg, op, in, out, ctx->s);
    count(ctx, mg_launches_per_cycle(ctx->mg, op.down0 != nullptr));
}

// the line preconditioner at U (1D, FP64)
m1_status build_line(m1_ctx* ctx, const Dev<double>& g, const double* U) {
    const size_t nu2 = (size_t)ctx->nu * ctx->nu;
    CKS(dalloc(ctx, &ctx->line_B, 3 * nu2 * ctx->N));
    CKS(dalloc(ctx, &ctx->line_M, nu2 * ctx->N));
    CKS(dalloc(ctx, &ctx->line_Dinv, nu2 * ctx->N));
    TK t(ctx, M1_K_PC_BUILD);
    CK(cudaMemsetAsync(ctx->singular, 0, sizeof(int), ctx->s));
    launch_line_build(g, U, ctx->line_B, ctx->line_M, ctx->line_Dinv, ctx->singular, ctx->s);
    count(ctx, 2);
    ctx->st.precond_builds++;
    return M1_OK;
}

m1_status build_precond(m1_ctx* ctx, const Dev<double>& g, const double* U) {
    TK t(ctx, M1_K_PC_BUILD);
    launch_diag_f64(g, U, ctx->blocks, ctx->s);
    CK(cudaMemsetAsync(ctx->singular, 0, sizeof(int), ctx->s));
    launch_block_inverse(ctx->nu, ctx->N, ctx->blocks, ctx->binv, ctx->binv32, ctx->singular, ctx->s);
    count(ctx, 2);
    ctx->st.precond_builds++;
    return M1_OK;
}

// ---------------------------------------------------------------- GMRES
// Precision-generic pieces of restarted right-preconditioned GMRES with CGS2
// Arnoldi (two classical Gram-Schmidt passes), FP64 dot accumulation and an
// FP64 Hessenberg least-squares solved by Givens rotations on the device.
struct Ops64 {
    m1_ctx* ctx;
    Dev<double> g;
    const double* U;
    bool precond;
    int step = 0;                // Arnoldi step of the next M application (unused: M is fixed)
    const double* pj = nullptr;  // dP/dU at U: J v as a linear stencil, else by dual numbers
    bool line = false;           // M^-1: the block-tridiagonal line solve instead of point-block Jacobi
    bool fused() const { return false; }
    void AM(const double*, double*) {}
    void A(const double* in, double* out) {
        TK t(ctx, M1_K_JV64);
        if (pj)
            launch_jv_linear_f64(g, U, pj, in, out, ctx->s);
        else
            jv_f64(g, U, in, out, ctx->s);
        count(ctx, 1);
        ctx->st.jv_calls++;
    }
    void M(const double* in, double* out) {
        TK t(ctx, M1_K_PC_APPLY);
        if (line) {
            launch_line_solve(ctx->nu, ctx->N, ctx->line_B, ctx->line_M, ctx->line_Dinv, in, out, ctx->s);
        } else if (precond) {
            launch_bj_apply_f64(ctx->nu, ctx->N, ctx->binv, in, out, ctx->s);
        } else {
            cudaMemcpyAsync(out, in, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s);
        }
        count(ctx, 1);
    }
};
struct Ops32 {
    m1_ctx* ctx;
    Dev<float> g;
    const float* U;
    bool precond;
    bool learned = false;
    int form = 0;               // the learned correction's form (m1_set_learned_form)
    int step = 0;               // Arnoldi step of the next M application (the learned correction: odd steps)
    const float* pj = nullptr;  // dP/dU at U in FP32: J v as a linear stencil, else by dual numbers
    bool mg = false;            // M^-1: one multigrid cycle instead of point-block Jacobi
    // J M^-1 v in one stencil (point-block Jacobi applied while staging)
    bool fused() const { return pj && precond && !learned && !mg; }
    void AM(const float* in, float* out) {
        TK t(ctx, M1_K_JV32);
        launch_jv_linear_pre_f32(g, U, pj, ctx->binv32, in, out, ctx->s);
        count(ctx, 1);
        ctx->st.jv_calls++;
    }
    void A(const float* in, float* out) {
        TK t(ctx, M1_K_JV32);
        if (pj)
            launch_jv_linear_f32(g, U, pj, in, out, ctx->s);
        else
            jv_f32(g, U, in, out, ctx->s);
        count(ctx, 1);
        ctx->st.jv_calls++;
    }
    void M(const float* in, float* out) {
        TK t(ctx, M1_K_PC_APPLY);
        if (mg) {
            mg_apply(ctx, in, out);
            return;
        }
        if (precond) {
            launch_bj_apply_f32(ctx->nu, ctx->N, ctx->binv32, in, out, ctx->s);
        } else {
            cudaMemcpyAsync(out, in, sizeof(float) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s);
        }
        count(ctx, 1);
        // + s (N(v / s) - N(0)) on odd Arnoldi steps: the Krylov vectors have unit norm,
        // s = 1 / sqrt(n); even steps keep the plain point-block Jacobi direction in the
        // flexible basis, so the learned directions can only add to it
        if (learned && form == M1_LEARNED_ADDITIVE && (step & 1)) {
            nn_apply_add(ctx->nn, in, ctx->N, ctx->nn_static, ctx->nn_null, (float)(1.0 / sqrt((double)ctx->n)), out,
                         ctx->s);
            count(ctx, 24);
        }
        // two-stage form: out = z1 = M^-1 v from above; r1 = v - J z1 is what point-block
        // Jacobi leaves, and out += M^-1 r1 + s1 (N(r1 / s1) - N(0)), s1 the RMS of r1:
        // the network sees the residual of a point-block Jacobi stage, the input it is
        // trained on (J e for the errors point-block Jacobi resolves slowly)
        if (learned && form != M1_LEARNED_ADDITIVE && (form == M1_LEARNED_TWO_STAGE_ALL || (step & 1))) {
            cudaStream_t s = ctx->s;
            if (pj)
                launch_jv_linear_f32(g, U, pj, out, ctx->nn_r, s);
            else
                jv_f32(g, U, out, ctx->nn_r, s);
            launch_axpby_f32(1.f, in, -1.f, ctx->nn_r, ctx->nn_r, ctx->n, s);
            launch_bj_apply_f32(ctx->nu, ctx->N, ctx->binv32, ctx->nn_r, ctx->nn_t, s);
            launch_axpby_f32(1.f, ctx->nn_t, 1.f, out, out, ctx->n, s);
            launch_norm2_f32(ctx->nn_r, ctx->n, ctx->nn_part, ctx->nn_n2, s);
            nn_apply_add_rms(ctx->nn, ctx->nn_r, ctx->N, ctx->nn_static, ctx->nn_null, ctx->nn_n2, out, s);
            count(ctx, 30);
            ctx->st.jv_calls++;
        }
    }
};

ArnoldiDev arnoldi_dev(m1_ctx* ctx, bool fp32) {
    ArnoldiDev K;
    K.n = ctx->n;
    K.ld = ctx->ld;
    const int* grid = fp32 ? ctx->gs_grid32 : ctx->gs_grid64;
    const int* grid_dots = fp32 ? ctx->gs_dots32 : ctx->gs_dots64;
    for (int j = 0; j < kMaxRestart; ++j) {
        K.grid[j] = grid[j];
        K.grid_dots[j] = grid_dots[j];
    }
    K.H = ctx->sc.H;
    K.cs = ctx->sc.cs;
    K.sn = ctx->sc.sn;
    K.g = ctx->sc.g;
    K.resid = ctx->sc.resid;
    K.h1 = ctx->sc.h1;
    K.h2 = ctx->sc.h2;
    K.nrm2 = ctx->sc.nrm2;
    K.partials = ctx->ar_partials;
    K.partials2 = ctx->ar_partials + (size_t)kMaxGsBlocks * (kPartCols + 1);
    K.reorth = ctx->ar_reorth;
    K.resid_host = nullptr;
    return K;
}
inline void arnoldi_step(const ArnoldiDev& K, double* V, double* w, int j, cudaStream_t s) {
    launch_arnoldi_step_f64(K, V, w, j, s);
}
inline void arnoldi_step(const ArnoldiDev& K, float* V, float* w, int j, cudaStream_t s) {
    launch_arnoldi_step_f32(K, V, w, j, s);
}

inline void scale_inv_sqrt(const double* x, const double* n2, double* y, long long n, cudaStream_t s) {
    launch_scale_inv_sqrt_f64(x, n2, y, n, s);
}
inline void scale_inv_sqrt(const float* x, const double* n2, float* y, long long n, cudaStream_t s) {
    launch_scale_inv_sqrt_f32(x, n2, y, n, s);
}
inline void lincomb_add(const double* Z, long long ld, int k, const double* y, double* x, long long n,
                        cudaStream_t s) {
    launch_lincomb_add_f64(Z, ld, k, y, x, n, s);
}
inline void lincomb_add(const float* Z, long long ld, int k, const double* y, double* x, long long n,
                        cudaStream_t s) {
    launch_lincomb_add_f32_to_f64(Z, ld, k, y, x, n, s);
}
inline void norm2(const double* x, long long n, double* p, double* out, cudaStream_t s) {
    launch_norm2_f64(x, n, p, out, s);
}
inline void norm2(const float* x, long long n, double* p, double* out, cudaStream_t s) {
    launch_norm2_f32(x, n, p, out, s);
}

// One GMRES(m) cycle on A M^-1 from the residual r0 (||r0||^2 in sc.nrm2[0],
// ||r0|| = beta). On return ctx->tmp (FP64) holds V y, the caller adds
// M^-1 V y to its solution. *kout = Arnoldi steps taken, *est = the final
// residual estimate |g_k|.
template <class T, class Ops>
m1_status gmres_cycle(m1_ctx* ctx, Ops& ops, T* V, T* w, T* z, const T* r0, double beta, double target, int maxk,
                      int* kout, double* est, T* Z = nullptr) {
    const long long n = ctx->n;
    cudaStream_t s = ctx->s;
    const Scal& sc = ctx->sc;
    scale_inv_sqrt(r0, sc.nrm2, V, n, s);
    count(ctx, 1);
    std::vector<double> g0(kPartCols, 0.0);
    g0[0] = beta;
    CK(cudaMemcpyAsync(sc.g, g0.data(), sizeof(double) * kPartCols, cudaMemcpyHostToDevice, s));
    int k = 0;
    double e = beta;
    const long long ld = ctx->ld;
    // Step j is enqueued before the host reads the residual estimate of step
    // j - 1, so the device never idles on the convergence test. A step enqueued
    // past the stopping one is discarded: it writes only V_{j+1}, z_j,
    // Hessenberg column j, the rotation j and g[j], g[j+1], none of which the
    // back substitution over the first j columns reads.
    for (int j = 0; j <= maxk; ++j) {
        if (j < maxk) {
            T* Vj = V + (long long)j * ld;
            if (!Z && ops.fused()) {
                ops.AM(Vj, w);  // J M^-1 V_j, M^-1 V_j never stored
            } else {
                T* zj = Z ? Z + (long long)j * ld : z;  // flexible GMRES keeps every preconditioned vector
                ops.step = j;
                ops.M(Vj, zj);
                ops.A(zj, w);
            }
            {
                TK t(ctx, M1_K_ORTHO);
                // the update pass writes step j's estimate straight into the
                // mapped host slot; without mapping it is copied after the pass
                ArnoldiDev K = arnoldi_dev(ctx, sizeof(T) == 4);
                K.resid_host = ctx->hpin_dev ? ctx->hpin_dev + 8 + 4 * (j & 1) : nullptr;
                arnoldi_step(K, V, w, j, s);
            }
            count(ctx, 3);
            if (!ctx->hpin_dev)
                CK(cudaMemcpyAsync(ctx->hpin + 8 + 4 * (j & 1), sc.resid, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                   s));
            CK(cudaEventRecord(ctx->ev_res[j & 1], s));
        }
        if (j == 0) continue;
        const int jj = j - 1;  // the step inspected now
        CK(cudaGetLastError());
        CK(cudaEventSynchronize(ctx->ev_res[jj & 1]));
        const double* r = ctx->hpin + 8 + 4 * (jj & 1);
        k = jj + 1;
        e = r[0];
        ctx->st.gmres_iters++;
        // the dots pass reads V_0..V_j and w (and once more for the second
        // Gram-Schmidt pass); the update reads them and writes V_{j+1}
        ctx->st.ortho_bytes += (double)sizeof(T) * n * ((jj + 2.0) * (1.0 + r[2]) + (jj + 3.0));
        if (!(e == e)) {
            cudaStreamSynchronize(s);
            return fail(ctx, M1_ERR_NONFINITE, "non-finite GMRES residual estimate");
        }
        if (e <= target || r[1] == 0.0) break;
    }
    launch_backsolve(sc.H, sc.g, k, sc.y, s);
    CK(cudaMemsetAsync(ctx->tmp, 0, sizeof(double) * n, s));
    lincomb_add(Z ? Z : V, ld, k, sc.y, ctx->tmp, n, s);  // flexible: tmp = Z y, else V y
    count(ctx, 2);
    *kout = k;
    *est = e;
    return M1_OK;
}

// Restarted right-preconditioned GMRES in FP64: x = J(U)^-1 b to rtol.
m1_status gmres64(m1_ctx* ctx, Ops64& ops, const double* b, double* x, double rtol, int restart, int maxit,
                  int* iters, double* bnorm_out, double* res_out, bool* conv) {
    const long long n = ctx->n;
    cudaStream_t s = ctx->s;
    double bnorm;
    CKS(norm_f64(ctx, b, &bnorm));
    *bnorm_out = bnorm;
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    *iters = 0;
    *conv = false;
    *res_out = bnorm;
    if (bnorm == 0.0) {
        *conv = true;
        return M1_OK;
    }
    if (!(bnorm == bnorm)) return fail(ctx, M1_ERR_NONFINITE, "non-finite right-hand side");
    const double target = rtol * bnorm;
    for (bool first = true;; first = false) {
        double beta;
        if (first) {  // x = 0: r = b, ||b||^2 already in sc.nrm2[0]
            CK(cudaMemcpyAsync(ctx->rhs, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            beta = bnorm;
        } else {  // r = b - J x
            ops.A(x, ctx->w);
            launch_axpby_f64(1.0, b, -1.0, ctx->w, ctx->rhs, n, s);
            count(ctx, 1);
            CKS(norm_f64(ctx, ctx->rhs, &beta));
        }
        *res_out = beta;
        if (!(beta == beta)) return fail(ctx, M1_ERR_NONFINITE, "non-finite GMRES residual");
        if (beta <= target) {
            *conv = true;
            return M1_OK;
        }
        if (*iters >= maxit) return M1_OK;
        int k;
        double est;
        const int maxk = std::min(restart, maxit - *iters);
        CKS(gmres_cycle<double>(ctx, ops, ctx->V, ctx->w, ctx->z, ctx->rhs, beta, target, maxk, &k, &est));
        *iters += k;
        ops.M(ctx->tmp, ctx->z);
        launch_axpy_f64(1.0, ctx->z, x, n, s);
        count(ctx, 1);
    }
}

// Mixed precision: FP32 inner GMRES (FP32 Jv, FP32 basis and block inverse,
// FP64 dot accumulation and Hessenberg) on r / ||r||, refined against the
// FP64 linear residual r = b - J x (FP64 Jv) until rtol is met.
// ---------------------------------------------------------------- BiCGStab
inline void bs_dots(const double* a0, const double* b0, const double* a1, const double* b1, long long n, int nd,
                    double* part, int mode, double* sc, double* slot, cudaStream_t s) {
    launch_bs_dots_f64(a0, b0, a1, b1, n, nd, part, mode, sc, slot, s);
}
inline void bs_dots(const float* a0, const float* b0, const float* a1, const float* b1, long long n, int nd,
                    double* part, int mode, double* sc, double* slot, cudaStream_t s) {
    launch_bs_dots_f32(a0, b0, a1, b1, n, nd, part, mode, sc, slot, s);
}
inline void bs_p(double* p, const double* r, const double* v, const double* sc, long long n, cudaStream_t s) {
    launch_bs_p_f64(p, r, v, sc, n, s);
}
inline void bs_p(float* p, const float* r, const float* v, const double* sc, long long n, cudaStream_t s) {
    launch_bs_p_f32(p, r, v, sc, n, s);
}
inline void bs_s(double* sv, const double* r, const double* v, const double* sc, long long n, cudaStream_t s) {
    launch_bs_s_f64(sv, r, v, sc, n, s);
}
inline void bs_s(float* sv, const float* r, const float* v, const double* sc, long long n, cudaStream_t s) {
    launch_bs_s_f32(sv, r, v, sc, n, s);
}
inline void bs_xr(double* x, double* r, const double* ph, const double* sh, const double* sv, const double* t,
                  const double* rh, double* sc, long long n, double* part, double* slot, cudaStream_t s) {
    launch_bs_xr_f64(x, r, ph, sh, sv, t, rh, sc, n, part, slot, s);
}
inline void bs_xr(double* x, float* r, const float* ph, const float* sh, const float* sv, const float* t,
                  const float* rh, double* sc, long long n, double* part, double* slot, cudaStream_t s) {
    launch_bs_xr_f32(x, r, ph, sh, sv, t, rh, sc, n, part, slot, s);
}

// Right-preconditioned BiCGStab (Sect. 3.3.1) on A M^-1 from x = 0: x (FP64) +=
// the solution of A x = b to ||r|| <= target; the eight work vectors are rows of
// `work` (stride ld). The host reads ||r||^2 and the breakdown flag once per
// iteration (every scalar of the recurrence stays on the device).
template <class T, class Ops>
m1_status bicgstab_solve(m1_ctx* ctx, Ops& ops, const T* b, double* x, double target, int maxit, T* work,
                         int* iters, double* res_out, bool* conv) {
    const long long n = ctx->n, ld = ctx->ld;
    cudaStream_t s = ctx->s;
    CKS(dalloc(ctx, &ctx->bs_part, (size_t)bs_partial_rows()));
    CKS(dalloc(ctx, &ctx->bs_sc, (size_t)kBsScalars));
    T *r = work, *rh = work + ld, *p = work + 2 * ld, *v = work + 3 * ld, *ph = work + 4 * ld, *sv = work + 5 * ld,
      *sh = work + 6 * ld, *t = work + 7 * ld;
    CK(cudaMemcpyAsync(r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(rh, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(p, 0, sizeof(T) * n, s));
    CK(cudaMemsetAsync(v, 0, sizeof(T) * n, s));
    const double init[kBsScalars] = {1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // rho, alpha, omega
    CK(cudaMemcpyAsync(ctx->bs_sc, init, sizeof(init), cudaMemcpyHostToDevice, s));
    double* slot = ctx->hpin_dev ? ctx->hpin_dev + 8 : nullptr;
    auto read_slot = [&](double* rr, double* brk) -> m1_status {
        if (!slot) {
            CK(cudaMemcpyAsync(ctx->hpin + 8, ctx->bs_sc + kBsRR, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(ctx->hpin + 9, ctx->bs_sc + kBsBreak, sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        CK(cudaEventRecord(ctx->ev_res[0], s));
        CK(cudaGetLastError());
        CK(cudaEventSynchronize(ctx->ev_res[0]));
        *rr = ctx->hpin[8];
        *brk = ctx->hpin[9];
        return M1_OK;
    };
    {
        TK tk(ctx, M1_K_ORTHO);
        bs_dots(rh, r, r, r, n, 2, ctx->bs_part, kBsModeRho, ctx->bs_sc, slot, s);  // rho = (rhat, r), ||r||^2
    }
    count(ctx, 2);
    double rr, brk;
    CKS(read_slot(&rr, &brk));
    *iters = 0;
    *conv = sqrt(rr) <= target;
    *res_out = sqrt(rr);
    while (!*conv && *iters < maxit) {
        {
            TK tk(ctx, M1_K_VECTOR);
            bs_p(p, r, v, ctx->bs_sc, n, s);
        }
        ops.M(p, ph);
        ops.A(ph, v);
        {
            TK tk(ctx, M1_K_ORTHO);
            bs_dots(rh, v, (const T*)nullptr, (const T*)nullptr, n, 1, ctx->bs_part, kBsModeAlpha, ctx->bs_sc,
                    nullptr, s);
        }
        {
            TK tk(ctx, M1_K_VECTOR);
            bs_s(sv, r, v, ctx->bs_sc, n, s);
        }
        ops.M(sv, sh);
        ops.A(sh, t);
        {
            TK tk(ctx, M1_K_ORTHO);
            bs_dots(t, sv, t, t, n, 2, ctx->bs_part, kBsModeOmega, ctx->bs_sc, nullptr, s);
            bs_xr(x, r, ph, sh, sv, t, rh, ctx->bs_sc, n, ctx->bs_part, slot, s);
        }
        count(ctx, 8);
        CKS(read_slot(&rr, &brk));
        ++*iters;
        ctx->st.gmres_iters++;
        if (!(rr == rr)) return fail(ctx, M1_ERR_NONFINITE, "non-finite BiCGStab residual");
        *res_out = sqrt(rr);
        *conv = *res_out <= target;
        if (brk != 0.0) break;  // a zero denominator: stop with the iterate reached
    }
    return M1_OK;
}

m1_status gmres_mixed(m1_ctx* ctx, Ops64& ops64, Ops32& ops32, const double* b, double* x, double rtol,
                      int restart, int maxit, int refine_max, int* iters, int* refinements, double* bnorm_out,
                      double* res_out, bool* conv, bool bicg = false) {
    const bool flexible = ops32.learned;
    const long long n = ctx->n;
    cudaStream_t s = ctx->s;
    double bnorm;
    CKS(norm_f64(ctx, b, &bnorm));  // leaves ||b||^2 in sc.nrm2[0]
    *bnorm_out = bnorm;
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    *iters = 0;
    *refinements = 0;
    *conv = false;
    *res_out = bnorm;
    if (bnorm == 0.0) {
        *conv = true;
        return M1_OK;
    }
    const double target = rtol * bnorm;
    CK(cudaMemcpyAsync(ctx->rhs, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double rnorm = bnorm;
    for (int sweep = 0;; ++sweep) {
        *res_out = rnorm;
        if (!(rnorm == rnorm)) return fail(ctx, M1_ERR_NONFINITE, "non-finite refinement residual");
        if (rnorm <= target) {
            *conv = true;
            return M1_OK;
        }
        if (sweep > refine_max || *iters >= maxit) return M1_OK;
        // inner relative tolerance that meets the outer target if FP32 were exact
        const double inner_rtol = std::max(0.5 * target / rnorm, 1e-6);
        launch_scale_f64_to_f32(ctx->rhs, ctx->sc.nrm2, ctx->w32, n, s);  // unit right-hand side
        CK(cudaMemsetAsync(ctx->xacc, 0, sizeof(double) * n, s));
        count(ctx, 1);
        if (bicg) {  // FP32 BiCGStab on the unit right-hand side, its iterate accumulated in FP64
            int k = 0;
            double est = 0.0;
            bool c = false;
            CKS(bicgstab_solve<float>(ctx, ops32, ctx->w32, ctx->xacc, inner_rtol, maxit - *iters, ctx->V32, &k, &est,
                                      &c));
            *iters += k;
        }
        for (bool first = true; !bicg; first = false) {
            // r32 = unit rhs - J32 xacc
            if (first) {
                CK(cudaMemcpyAsync(ctx->tmp32, ctx->w32, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
            } else {
                launch_f64_to_f32(ctx->xacc, ctx->z32, n, s);
                ops32.A(ctx->z32, ctx->tmp32);
                launch_f32_to_f64(ctx->tmp32, ctx->tmp, n, s);
                launch_f32_to_f64(ctx->w32, ctx->z, n, s);
                launch_axpby_f64(1.0, ctx->z, -1.0, ctx->tmp, ctx->tmp, n, s);
                launch_f64_to_f32(ctx->tmp, ctx->tmp32, n, s);
                count(ctx, 4);
            }
            launch_norm2_f32(ctx->tmp32, n, ctx->partials, ctx->sc.nrm2, s);
            count(ctx, 2);
            CK(cudaMemcpyAsync(ctx->hpin, ctx->sc.nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
            CKS(sync(ctx));
            const double beta = sqrt(ctx->hpin[0]);
            if (!(beta == beta)) return fail(ctx, M1_ERR_NONFINITE, "non-finite inner residual");
            if (beta <= inner_rtol || *iters >= maxit) break;
            int k;
            double est;
            const int maxk = std::min(restart, maxit - *iters);
            CKS(gmres_cycle<float>(ctx, ops32, ctx->V32, ctx->z32 /*w*/, ctx->tmp32 /*z*/, ctx->tmp32, beta,
                                   inner_rtol, maxk, &k, &est, flexible ? ctx->Z32 : nullptr));
            *iters += k;
            if (flexible) {  // tmp = Z y already holds the preconditioned combination
                launch_axpy_f64(1.0, ctx->tmp, ctx->xacc, n, s);
            } else if (ops32.mg) {  // M^-1 (V y): the same FP32 cycle the Krylov space used
                launch_f64_to_f32(ctx->tmp, ctx->tmp32, n, s);
                ops32.M(ctx->tmp32, ctx->z32);
                launch_f32_to_f64(ctx->z32, ctx->z, n, s);
                launch_axpy_f64(1.0, ctx->z, ctx->xacc, n, s);
                count(ctx, 2);
            } else {
                ops64.M(ctx->tmp, ctx->z);
                launch_axpy_f64(1.0, ctx->z, ctx->xacc, n, s);
            }
            count(ctx, 1);
        }
        // x += ||r|| xacc ; r = b - J64 x
        launch_axpy_f64(rnorm, ctx->xacc, x, n, s);
        ops64.A(x, ctx->w);
        launch_axpby_f64(1.0, b, -1.0, ctx->w, ctx->rhs, n, s);
        count(ctx, 2);
        CKS(norm_f64(ctx, ctx->rhs, &rnorm));  // leaves ||r||^2 in sc.nrm2[0]
        ++*refinements;
    }
}

m1_status validate(const m1_grid_desc* d, std::string& why) {
    if (!d) {
        why = "null descriptor";
        return M1_ERR_ARG;
    }
    if (d->dim < 1 || d->dim > 3) {
        why = "dim must be 1, 2 or 3";
        return M1_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        if (d->n[a] < 1) {
            why = "n[a] must be >= 1";
            return M1_ERR_ARG;
        }
        if (a >= d->dim && d->n[a] != 1) {
            why = "unused axes must have n = 1";
            return M1_ERR_ARG;
        }
        if (a < d->dim) {
            if (!(d->hi[a] > d->lo[a])) {
                why = "hi must exceed lo";
                return M1_ERR_ARG;
            }
            for (int sd = 0; sd < 2; ++sd)
                if (d->bc[a][sd] < 0 || d->bc[a][sd] > 3) {
                    why = "unknown boundary kind";
                    return M1_ERR_ARG;
                }
            if ((d->bc[a][0] == M1_BC_PERIODIC) != (d->bc[a][1] == M1_BC_PERIODIC)) {
                why = "periodic must be set on both sides of an axis";
                return M1_ERR_ARG;
            }
        }
    }
    if (!(d->c > 0.0) || !(d->a_r > 0.0)) {
        why = "c and a_r must be positive";
        return M1_ERR_ARG;
    }
    if (!(d->lambda_floor >= 0.0)) {
        why = "lambda_floor must be >= 0";
        return M1_ERR_ARG;
    }
    const long long N = (long long)d->n[0] * d->n[1] * d->n[2];
    if (N > (1LL << 31)) {
        why = "grid too large";
        return M1_ERR_ARG;
    }
    return M1_OK;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

void m1_default_opts(m1_solver_opts* o) {
    if (!o) return;
    o->newton_rtol = 1e-8;
    o->newton_max = 30;
    o->restart = 30;
    o->gmres_max = 3000;
    o->gmres_rtol = 1e-4;
    o->precision = M1_PREC_FP64;
    o->precond = M1_PRECOND_BJ;
    o->line_search = 1;
    o->advance = 1;
    o->refine_max = 4;
    o->krylov = M1_KRYLOV_GMRES;
    o->pc_rebuild = 1;
    o->realizability = 0;
    o->check_every = 5;
    o->forcing = 0;
}

m1_status m1_init_grid(const m1_grid_desc* desc, void* cuda_stream, m1_ctx** out) {
    if (!out) return M1_ERR_ARG;
    *out = nullptr;
    std::string why;
    m1_status v = validate(desc, why);
    if (v != M1_OK) return v;
    m1_ctx* ctx = new (std::nothrow) m1_ctx();
    if (!ctx) return M1_ERR_NOMEM;
    ctx->d = *desc;
    ctx->s = (cudaStream_t)cuda_stream;
    ctx->fp64_df = ctx->fp64_df_ok = fp64_auto_df(*desc);
    ctx->dim = desc->dim;
    ctx->nu = 1 + desc->dim + (desc->gas_coupling ? 1 : 0);
    ctx->N = (long long)desc->n[0] * desc->n[1] * desc->n[2];
    ctx->n = ctx->N * ctx->nu;
    ctx->ld = (ctx->n + 63) / 64 * 64;
    for (int a = 0; a < 3; ++a) {
        ctx->nfaces[a] = ctx->N / desc->n[a] * (desc->n[a] + 1);
        ctx->bM[a] = ctx->N / desc->n[a];
    }
    auto cleanup = [&](m1_status st) {
        ctx->err.clear();
        m1_destroy(ctx);
        return st;
    };
    const long long N = ctx->N, n = ctx->n;
#define AL(p, cnt)                                        \
    do {                                                  \
        m1_status st_ = dalloc(ctx, &(p), (size_t)(cnt)); \
        if (st_ != M1_OK) return cleanup(st_);            \
    } while (0)
    AL(ctx->sig_a, N);
    AL(ctx->sig_f, N);
    AL(ctx->Un, n);
    AL(ctx->Unew, n);
    AL(ctx->sig_a32, N);
    AL(ctx->sig_f32, N);
    AL(ctx->Un32, n);
    if (desc->gas_coupling) {
        AL(ctx->rho_cv, N);
        AL(ctx->rho_cv32, N);
    } else {
        AL(ctx->B, N);
        AL(ctx->B32, N);
    }
    for (int a = 0; a < ctx->dim; ++a) {
        AL(ctx->f64.alpha[a], ctx->nfaces[a]);
        AL(ctx->f64.lam_p[a], ctx->nfaces[a]);
        AL(ctx->f64.lam_m[a], ctx->nfaces[a]);
        AL(ctx->f32.alpha[a], ctx->nfaces[a]);
        AL(ctx->f32.lam_p[a], ctx->nfaces[a]);
        AL(ctx->f32.lam_m[a], ctx->nfaces[a]);
    }
    ctx->residual_partials = std::max((long long)reduce_blocks() * kPartCols, residual_partial_count(ctx->dim, ctx->d.n));
    AL(ctx->partials, (size_t)ctx->residual_partials);
    const size_t nscal = 4 + 4 * kPartCols + (size_t)kHLd * kMaxRestart + 2 * kMaxRestart + 4;
    AL(ctx->scal_base, nscal);
    AL(ctx->singular, 1);
    AL(ctx->viol, 1);
    AL(ctx->ar_partials, (size_t)2 * kMaxGsBlocks * (kPartCols + 1));
    AL(ctx->ar_reorth, 1);
#undef AL
    double* p = ctx->scal_base;
    ctx->sc.nrm2 = p;
    p += 4;
    ctx->sc.h1 = p;
    p += kPartCols;
    ctx->sc.h2 = p;
    p += kPartCols;
    ctx->sc.g = p;
    p += kPartCols;
    ctx->sc.y = p;
    p += kPartCols;
    ctx->sc.H = p;
    p += (size_t)kHLd * kMaxRestart;
    ctx->sc.cs = p;
    p += kMaxRestart;
    ctx->sc.sn = p;
    p += kMaxRestart;
    ctx->sc.resid = p;
    if (cudaHostAlloc((void**)&ctx->hpin, 16 * sizeof(double), cudaHostAllocMapped) != cudaSuccess)
        return cleanup(M1_ERR_NOMEM);
    if (cudaHostGetDevicePointer((void**)&ctx->hpin_dev, ctx->hpin, 0) != cudaSuccess) {
        ctx->hpin_dev = nullptr;  // fall back to copies
        cudaGetLastError();
    }
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_res[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_res[1], cudaEventDisableTiming) != cudaSuccess)
        return cleanup(M1_ERR_CUDA);
    if (cudaMemsetAsync(ctx->scal_base, 0, nscal * sizeof(double), ctx->s) != cudaSuccess) return cleanup(M1_ERR_CUDA);
    if (cudaMemsetAsync(ctx->ar_reorth, 0, sizeof(int), ctx->s) != cudaSuccess)
        return cleanup(M1_ERR_CUDA);
    if (!desc->gas_coupling && cudaMemsetAsync(ctx->B, 0, N * sizeof(double), ctx->s) != cudaSuccess)
        return cleanup(M1_ERR_CUDA);
    if (cudaStreamSynchronize(ctx->s) != cudaSuccess) return cleanup(M1_ERR_CUDA);
    arnoldi_grid_table(ctx->n, true, ctx->gs_grid32, ctx->gs_dots32);
    arnoldi_grid_table(ctx->n, false, ctx->gs_grid64, ctx->gs_dots64);
    if (cudaGetLastError() != cudaSuccess) return cleanup(M1_ERR_CUDA);
    {
        // minimal traffic per launch: J v reads U, v, sigma_a, sigma_f, alpha (one
        // face per cell and axis), the time-n wave speeds when they are frozen
        // (two per face), rho c_v with gas; writes J v. The residual also reads
        // U^n and the emission (or T^n) and the source.
        const double nu = ctx->nu, dim = ctx->dim;
        const double fields = 2.0 + dim + (desc->implicit_eigs ? 0.0 : 2.0 * dim) + (desc->gas_coupling ? 1.0 : 0.0);
        // the linear 2D J v reads v and dP/dU (9 planes, + d(a_r T^4)/dT with
        // gas) instead of U and v; the FP32 one also reads the n_u x n_u block
        // inverse it applies while staging (J M^-1 v)
        const bool lin = desc->dim == 2 && (desc->fixed_eigs || !desc->implicit_eigs);
        const double jv_fields = lin ? 2.0 * nu + fields + 9.0 + (desc->gas_coupling ? 1.0 : 0.0) : 3.0 * nu + fields;
        ctx->st.bytes_per_jv = (double)N * 8.0 * jv_fields;
        ctx->st.bytes_per_jv32 = (double)N * 4.0 * (jv_fields + (lin ? nu * nu : 0.0));
        ctx->st.bytes_per_residual = (double)N * 8.0 * (3.0 * nu + fields + (desc->gas_coupling ? 0.0 : 1.0));
    }
    *out = ctx;
    return M1_OK;
}

m1_status m1_destroy(m1_ctx* ctx) {
    if (!ctx) return M1_OK;
    cudaStreamSynchronize(ctx->s);
    void* ptrs[] = {ctx->sig_a, ctx->sig_f, ctx->B, ctx->S, ctx->rho_cv, ctx->Un, ctx->Unew, ctx->sig_a32,
                    ctx->sig_f32, ctx->B32, ctx->S32, ctx->rho_cv32, ctx->Un32, ctx->U, ctx->R, ctx->Ut, ctx->Rt,
                    ctx->delta, ctx->rhs, ctx->w, ctx->z, ctx->tmp, ctx->V, ctx->xacc, ctx->blocks, ctx->binv,
                    ctx->binv32, ctx->V32, ctx->w32, ctx->z32, ctx->U32, ctx->tmp32, ctx->Fstar, ctx->linework,
                    ctx->partials, ctx->scal_base, ctx->singular, ctx->viol, ctx->ar_partials,
                    ctx->ar_reorth, ctx->logsig, ctx->nn_static, ctx->nn_null, ctx->Z32, ctx->pair_x, ctx->pair_t, ctx->pj64, ctx->pj32, ctx->bs_part, ctx->bs_sc,
                    ctx->fb, ctx->fbw, ctx->nn_r, ctx->nn_t, ctx->nn_part, ctx->nn_n2};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (int l = 0; l < kMgMaxLevels; ++l) {
        for (float* q : {ctx->mg.A[l], ctx->mg.r[l], ctx->mg.z[l], ctx->mg.z2[l]})
            if (q) cudaFree(q);
        if (l > 0 && ctx->mg.Dinv[l]) cudaFree(ctx->mg.Dinv[l]);
    }
    for (void* q : {(void*)ctx->mg.w0, (void*)ctx->mg.probe, (void*)ctx->mg_inv64, (void*)ctx->line_B,
                    (void*)ctx->line_M, (void*)ctx->line_Dinv})
        if (q) cudaFree(q);
    for (int a = 0; a < 3; ++a) {
        void* fp[] = {ctx->f64.alpha[a], ctx->f64.lam_p[a], ctx->f64.lam_m[a],
                      ctx->f32.alpha[a], ctx->f32.lam_p[a], ctx->f32.lam_m[a]};
        for (void* q : fp)
            if (q) cudaFree(q);
        for (int sd = 0; sd < 2; ++sd) {
            void* bp[] = {ctx->bE[a][sd], ctx->bF[a][sd], ctx->bmask[a][sd], ctx->bE32[a][sd], ctx->bF32[a][sd]};
            for (void* q : bp)
                if (q) cudaFree(q);
        }
    }
    for (int a = 0; a < 3; ++a)
        if (ctx->vel[a]) cudaFree(ctx->vel[a]);
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t ev : ctx->ev_res)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t e : ctx->evs) cudaEventDestroy(e);
    delete ctx;
    return M1_OK;
}

m1_status m1_set_opacity(m1_ctx* ctx, const double* sigma_a, const double* sigma_f, m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    if (!sigma_a) return fail(ctx, M1_ERR_ARG, "sigma_a is required");
    const size_t bytes = sizeof(double) * ctx->N;
    CKS(copy_in(ctx, ctx->sig_a, sigma_a, bytes, mem));
    CKS(copy_in(ctx, ctx->sig_f, sigma_f ? sigma_f : sigma_a, bytes, mem));
    ctx->has_opacity = true;
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_set_state(m1_ctx* ctx, const double* E, const double* F, const double* T, const double* rho_cv,
                       m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    if (!E || !F) return fail(ctx, M1_ERR_ARG, "E and F are required");
    const bool gas = ctx->d.gas_coupling != 0;
    if (gas && (!T || !rho_cv)) return fail(ctx, M1_ERR_ARG, "gas coupling needs T and rho_cv");
    if (!gas && (T || rho_cv)) return fail(ctx, M1_ERR_ARG, "T/rho_cv given without gas coupling");
    const size_t fb = sizeof(double) * ctx->N;
    CKS(copy_in(ctx, ctx->Un, E, fb, mem));
    CKS(copy_in(ctx, ctx->Un + ctx->N, F, fb * ctx->dim, mem));
    if (gas) {
        CKS(copy_in(ctx, ctx->Un + (1 + ctx->dim) * ctx->N, T, fb, mem));
        CKS(copy_in(ctx, ctx->rho_cv, rho_cv, fb, mem));
    }
    ctx->has_state = true;
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_get_state(const m1_ctx* cctx, double* E, double* F, double* T, m1_mem mem) {
    m1_ctx* ctx = const_cast<m1_ctx*>(cctx);
    if (!ctx) return M1_ERR_ARG;
    if (!ctx->has_state) return fail(ctx, M1_ERR_STATE, "no state");
    const size_t fb = sizeof(double) * ctx->N;
    if (E) CKS(copy_out(ctx, E, ctx->Un, fb, mem));
    if (F) CKS(copy_out(ctx, F, ctx->Un + ctx->N, fb * ctx->dim, mem));
    if (T && ctx->d.gas_coupling) CKS(copy_out(ctx, T, ctx->Un + (1 + ctx->dim) * ctx->N, fb, mem));
    return sync(ctx);
}

m1_status m1_get_solution(const m1_ctx* cctx, double* U, m1_mem mem) {
    m1_ctx* ctx = const_cast<m1_ctx*>(cctx);
    if (!ctx || !U) return M1_ERR_ARG;
    CKS(copy_out(ctx, U, ctx->Unew, sizeof(double) * ctx->n, mem));
    return sync(ctx);
}

m1_status m1_set_boundary(m1_ctx* ctx, int axis, int side, const double* E, const double* F,
                          const unsigned char* mask, m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    if (axis < 0 || axis >= ctx->dim || side < 0 || side > 1) return fail(ctx, M1_ERR_ARG, "bad axis/side");
    if (ctx->d.bc[axis][side] != M1_BC_DIRICHLET) return fail(ctx, M1_ERR_ARG, "face is not Dirichlet");
    if (!E || !F) return fail(ctx, M1_ERR_ARG, "E and F are required");
    const long long M = ctx->bM[axis];
    CKS(dalloc(ctx, &ctx->bE[axis][side], M));
    CKS(dalloc(ctx, &ctx->bF[axis][side], M * ctx->dim));
    CKS(dalloc(ctx, &ctx->bE32[axis][side], M));
    CKS(dalloc(ctx, &ctx->bF32[axis][side], M * ctx->dim));
    CKS(copy_in(ctx, ctx->bE[axis][side], E, sizeof(double) * M, mem));
    CKS(copy_in(ctx, ctx->bF[axis][side], F, sizeof(double) * M * ctx->dim, mem));
    if (mask) {
        CKS(dalloc(ctx, &ctx->bmask[axis][side], M));
        CKS(copy_in(ctx, ctx->bmask[axis][side], mask, M, mem));
    } else if (ctx->bmask[axis][side]) {
        cudaFree(ctx->bmask[axis][side]);
        ctx->bmask[axis][side] = nullptr;
    }
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_set_emission(m1_ctx* ctx, const double* B, m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    if (ctx->d.gas_coupling) return fail(ctx, M1_ERR_ARG, "emission is a_r T^4 with gas coupling");
    if (!B) return fail(ctx, M1_ERR_ARG, "B is required");
    CKS(copy_in(ctx, ctx->B, B, sizeof(double) * ctx->N, mem));
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_set_source(m1_ctx* ctx, const double* S, m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    if (!S) {
        if (ctx->S) cudaFree(ctx->S);
        if (ctx->S32) cudaFree(ctx->S32);
        ctx->S = nullptr;
        ctx->S32 = nullptr;
        ctx->dirty = true;
        return M1_OK;
    }
    CKS(dalloc(ctx, &ctx->S, ctx->N));
    CKS(dalloc(ctx, &ctx->S32, ctx->N));
    CKS(copy_in(ctx, ctx->S, S, sizeof(double) * ctx->N, mem));
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_set_velocity(m1_ctx* ctx, const double* ux, const double* uy, const double* uz, m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    const double* u[3] = {ux, uy, uz};
    for (int a = 0; a < ctx->dim; ++a) {
        if (!u[a]) return fail(ctx, M1_ERR_ARG, "a velocity component is missing");
        CKS(dalloc(ctx, &ctx->vel[a], ctx->nfaces[a]));
        CKS(copy_in(ctx, ctx->vel[a], u[a], sizeof(double) * ctx->nfaces[a], mem));
    }
    return sync(ctx);
}

m1_status m1_advect(m1_ctx* ctx, double dt) {
    if (!ctx) return M1_ERR_ARG;
    if (!(dt > 0.0)) return fail(ctx, M1_ERR_ARG, "dt must be positive");
    if (!ctx->d.gas_coupling) return fail(ctx, M1_ERR_ARG, "advection needs gas coupling");
    if (!ctx->vel[0]) return fail(ctx, M1_ERR_STATE, "no velocity: call m1_set_velocity");
    CKS(prepare(ctx));
    Dev<double> g = dev64(ctx, dt);
    double* Tn = ctx->Un + (1 + ctx->dim) * ctx->N;
    double* Tnew = ctx->Unew + (1 + ctx->dim) * ctx->N;
    {
        TK t(ctx, M1_K_EXPLICIT);
        launch_advect(g, ctx->vel, Tnew, ctx->s);
        count(ctx, 1);
    }
    CK(cudaMemcpyAsync(Tn, Tnew, sizeof(double) * ctx->N, cudaMemcpyDeviceToDevice, ctx->s));
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_velocity_sources(m1_ctx* ctx, double dt) {
    if (!ctx) return M1_ERR_ARG;
    if (!(dt > 0.0)) return fail(ctx, M1_ERR_ARG, "dt must be positive");
    if (!ctx->vel[0]) return fail(ctx, M1_ERR_STATE, "no velocity: call m1_set_velocity");
    CKS(prepare(ctx));
    const Dev<double> g = dev64(ctx, dt);
    {
        TK t(ctx, M1_K_EXPLICIT);
        launch_velocity_sources(g, ctx->vel, ctx->Unew, ctx->s);
        count(ctx, 1);
    }
    CK(cudaMemcpyAsync(ctx->Un, ctx->Unew, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s));
    ctx->dirty = true;
    return sync(ctx);
}

m1_status m1_explicit_step(m1_ctx* ctx, double dt) {
    if (!ctx) return M1_ERR_ARG;
    if (!(dt > 0.0)) return fail(ctx, M1_ERR_ARG, "dt must be positive");
    CKS(prepare(ctx));
    if (!ctx->expl_ok) {
        CKS(dalloc(ctx, &ctx->Fstar, (size_t)ctx->dim * ctx->N));
        CKS(dalloc(ctx, &ctx->linework, (size_t)3 * ctx->N));
        ctx->expl_ok = true;
    }
    Dev<double> g = dev64(ctx, dt);
    {
        TK t(ctx, M1_K_EXPLICIT);
        launch_explicit_hyp(g, ctx->Unew, ctx->Fstar, ctx->s);
        count(ctx, 1);
        for (int b = 0; b < ctx->dim; ++b) {
            launch_wb_lines(g, b, ctx->Fstar, ctx->Unew + (1 + b) * ctx->N, ctx->linework, ctx->s);
            count(ctx, 1);
        }
    }
    CK(cudaMemcpyAsync(ctx->Un, ctx->Unew, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s));
    ctx->dirty = true;
    ctx->st.explicit_steps++;
    CKS(sync(ctx));
    return prepare(ctx);
}

m1_status m1_residual(m1_ctx* ctx, double dt, const double* U, double* R, m1_mem mem) {
    if (!ctx || !U || !R) return M1_ERR_ARG;
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    CKS(copy_in(ctx, ctx->U, U, sizeof(double) * ctx->n, mem));
    double nrm;
    CKS(residual_norm(ctx, dev64(ctx, dt), ctx->U, ctx->R, &nrm));
    CKS(copy_out(ctx, R, ctx->R, sizeof(double) * ctx->n, mem));
    return sync(ctx);
}

m1_status m1_jv(m1_ctx* ctx, double dt, const double* U, const double* v, double* Jv, int precision, m1_mem mem) {
    if (!ctx || !U || !v || !Jv) return M1_ERR_ARG;
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    CKS(copy_in(ctx, ctx->U, U, sizeof(double) * ctx->n, mem));
    CKS(copy_in(ctx, ctx->z, v, sizeof(double) * ctx->n, mem));
    // FP32: the operator the inner solver applies, a linear stencil of dP/dU at
    // U where available (2D, frozen or fixed wave speeds), else dual numbers
    bool lin = false;
    if (precision == M1_PREC_MIXED) {
        CKS(ensure_work32(ctx));
        launch_f64_to_f32(ctx->U, ctx->U32, ctx->n, ctx->s);
        launch_f64_to_f32(ctx->z, ctx->z32, ctx->n, ctx->s);
        CKS(pressure_jacobian32(ctx, dev64(ctx, dt), dev32(ctx, dt), ctx->U32, &lin));
        if (lin)
            launch_jv_linear_f32(dev32(ctx, dt), ctx->U32, ctx->pj32, ctx->z32, ctx->w32, ctx->s);
        else
            jv_f32(dev32(ctx, dt), ctx->U32, ctx->z32, ctx->w32, ctx->s);
        launch_f32_to_f64(ctx->w32, ctx->w, ctx->n, ctx->s);
        count(ctx, 4);
    } else {  // FP64: dual numbers (the refinement's operator), in the context's FP64 arithmetic
        jv_f64(dev64(ctx, dt), ctx->U, ctx->z, ctx->w, ctx->s);
        count(ctx, 1);
    }
    ctx->st.jv_calls++;
    CKS(copy_out(ctx, Jv, ctx->w, sizeof(double) * ctx->n, mem));
    return sync(ctx);
}

m1_status m1_mg_apply(m1_ctx* ctx, double dt, const double* U, const double* r, double* z, m1_mem mem) {
    if (!ctx || !r || !z) return M1_ERR_ARG;
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    CKS(ensure_work32(ctx));
    if (U)
        CKS(copy_in(ctx, ctx->U, U, sizeof(double) * ctx->n, mem));
    else
        CK(cudaMemcpyAsync(ctx->U, ctx->Un, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s));
    const Dev<double> g = dev64(ctx, dt);
    if (!mg_supported(ctx, g))
        return fail(ctx, M1_ERR_ARG,
                    "multigrid needs dim 2, frozen or fixed wave speeds and >= 3 cells along periodic axes");
    launch_f64_to_f32(ctx->U, ctx->U32, ctx->n, ctx->s);
    const Dev<float> g32 = dev32(ctx, dt);
    bool lin = false;
    CKS(pressure_jacobian32(ctx, g, g32, ctx->U32, &lin));
    CKS(build_mg(ctx, g32));
    CKS(copy_in(ctx, ctx->tmp, r, sizeof(double) * ctx->n, mem));
    launch_f64_to_f32(ctx->tmp, ctx->tmp32, ctx->n, ctx->s);
    mg_apply(ctx, ctx->tmp32, ctx->z32);
    launch_f32_to_f64(ctx->z32, ctx->w, ctx->n, ctx->s);
    count(ctx, 2);
    CKS(copy_out(ctx, z, ctx->w, sizeof(double) * ctx->n, mem));
    return sync(ctx);
}

m1_status m1_mg_blocks(m1_ctx* ctx, int level, int* nlev, double* out, m1_mem mem) {
    if (!ctx) return M1_ERR_ARG;
    if (!ctx->mg_alloc) return fail(ctx, M1_ERR_STATE, "no multigrid hierarchy built yet (m1_mg_apply)");
    if (nlev) *nlev = ctx->mg.nlev;
    if (!out) return M1_OK;
    if (level < 0 || level >= ctx->mg.nlev) return fail(ctx, M1_ERR_ARG, "level out of range");
    const size_t cnt = (size_t)5 * ctx->nu * ctx->nu * ctx->mg.nx[level] * ctx->mg.ny[level];
    // widened through the level-0 FP64 block scratch when it is large enough, else in pieces
    const size_t chunk = (size_t)ctx->nu * ctx->nu * ctx->N;
    for (size_t off = 0; off < cnt; off += chunk) {
        const size_t k = std::min(chunk, cnt - off);
        launch_f32_to_f64(ctx->mg.A[level] + off, ctx->blocks, (long long)k, ctx->s);
        CKS(copy_out(ctx, out + off, ctx->blocks, sizeof(double) * k, mem));
    }
    return sync(ctx);
}

m1_status m1_diag_blocks(m1_ctx* ctx, double dt, const double* U, double* blocks, m1_mem mem) {
    if (!ctx || !U || !blocks) return M1_ERR_ARG;
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    CKS(copy_in(ctx, ctx->U, U, sizeof(double) * ctx->n, mem));
    launch_diag_f64(dev64(ctx, dt), ctx->U, ctx->blocks, ctx->s);
    count(ctx, 1);
    CKS(copy_out(ctx, blocks, ctx->blocks, sizeof(double) * ctx->nu * ctx->nu * ctx->N, mem));
    return sync(ctx);
}

// newton_iter: the Newton step within an implicit step (-1 outside one: always rebuild)
static m1_status linear_solve(m1_ctx* ctx, double dt, const double* Ud, const double* b, double* x,
                              const m1_solver_opts* o, int newton_iter, int* iters, int* refinements, double* bnorm,
                              double* res, bool* conv) {
    const bool learned = o->precond == M1_PRECOND_LEARNED;
    const bool use_mg = o->precond == M1_PRECOND_MG;
    const bool line = o->precond == M1_PRECOND_LINE;
    const bool pre = o->precond == M1_PRECOND_BJ || learned || use_mg || line;
    if (line && (ctx->dim != 1 || o->precision != M1_PREC_FP64 || ctx->N < 3))
        return fail(ctx, M1_ERR_ARG, "M1_PRECOND_LINE needs dim 1, M1_PREC_FP64 and >= 3 cells");
    if (o->restart < 1 || o->restart > kMaxRestart)
        return fail(ctx, M1_ERR_ARG, "restart must be in [1, 30]");
    if (o->krylov != M1_KRYLOV_GMRES && o->krylov != M1_KRYLOV_BICGSTAB)
        return fail(ctx, M1_ERR_ARG, "unknown Krylov method");
    if (learned && o->krylov != M1_KRYLOV_GMRES)
        return fail(ctx, M1_ERR_ARG, "the learned preconditioner needs flexible GMRES");
    if (learned && (o->precision != M1_PREC_MIXED || !ctx->nn))
        return fail(ctx, M1_ERR_ARG, "the learned preconditioner needs M1_PREC_MIXED and m1_set_preconditioner");
    if (learned) CKS(dalloc(ctx, &ctx->Z32, (size_t)ctx->ld * (kMaxRestart + 1)));
    if (learned && ctx->nn_form != M1_LEARNED_ADDITIVE) {
        CKS(dalloc(ctx, &ctx->nn_r, (size_t)ctx->n));
        CKS(dalloc(ctx, &ctx->nn_t, (size_t)ctx->n));
        CKS(dalloc(ctx, &ctx->nn_part, (size_t)reduce_blocks()));
        CKS(dalloc(ctx, &ctx->nn_n2, 1));
    }
    Dev<double> g = dev64(ctx, dt);
    if (use_mg && (o->precision != M1_PREC_MIXED || !mg_supported(ctx, g)))
        return fail(ctx, M1_ERR_ARG,
                    "M1_PRECOND_MG needs M1_PREC_MIXED, dim 2, frozen or fixed wave speeds and >= 3 cells along "
                    "periodic axes");
    Ops64 ops{ctx, g, Ud, pre};
    bool lin = false;
    *refinements = 0;
    if (o->precision == M1_PREC_MIXED) {
        // the FP32 operator from dP/dU in FP32; the one FP64 J v per refinement
        // sweep stays on dual numbers (cheaper than an FP64 dP/dU per Newton step)
        CKS(ensure_work32(ctx));
        launch_f64_to_f32(Ud, ctx->U32, ctx->n, ctx->s);
        count(ctx, 1);
        const Dev<float> g32 = dev32(ctx, dt);
        CKS(pressure_jacobian32(ctx, g, g32, ctx->U32, &lin));
        if (pre && !use_mg) {  // FP32 point blocks, inverted in FP64 (multigrid takes them from its level 0)
            TK t(ctx, M1_K_PC_BUILD);
            launch_diag_f32(g32, ctx->U32, reinterpret_cast<float*>(ctx->blocks), ctx->s);
            CK(cudaMemsetAsync(ctx->singular, 0, sizeof(int), ctx->s));
            launch_block_inverse_f32(ctx->nu, ctx->N, reinterpret_cast<const float*>(ctx->blocks), ctx->binv,
                                     ctx->binv32, ctx->singular, ctx->s);
            count(ctx, 2);
            ctx->st.precond_builds++;
        }
        const int every = std::max(1, o->pc_rebuild);
        if (use_mg && (newton_iter < 0 || newton_iter % every == 0)) CKS(build_mg(ctx, g32));
        Ops32 ops32{ctx, g32, ctx->U32, pre};
        ops32.learned = learned;
        ops32.form = ctx->nn_form;
        if (learned) {  // the network's opacity and state planes at this Newton iterate, and its zero response
            launch_nn_static_f32(ctx->U32, ctx->N, ctx->d.c, ctx->logsig, ctx->nn_static, ctx->s);
            CK(cudaMemsetAsync(ctx->tmp32, 0, sizeof(float) * ctx->n, ctx->s));
            if (nn_null_response(ctx->nn, ctx->tmp32, ctx->N, ctx->nn_static, ctx->nn_null, ctx->s) != M1_OK)
                return fail(ctx, M1_ERR_CUDA, "learned preconditioner: null response failed");
            count(ctx, 23);
        }
        ops32.mg = use_mg;
        if (lin) ops32.pj = ctx->pj32;
        return gmres_mixed(ctx, ops, ops32, b, x, o->gmres_rtol, o->restart, o->gmres_max, o->refine_max, iters,
                           refinements, bnorm, res, conv, o->krylov == M1_KRYLOV_BICGSTAB);
    }
    CKS(pressure_jacobian64(ctx, g, Ud, &lin));
    if (lin) ops.pj = ctx->pj64;
    if (line) {
        CKS(build_line(ctx, g, Ud));
        ops.line = true;
    } else if (pre) {
        CKS(build_precond(ctx, g, Ud));
    }
    if (o->krylov == M1_KRYLOV_BICGSTAB) {
        double bn;
        CKS(norm_f64(ctx, b, &bn));
        *bnorm = bn;
        CK(cudaMemsetAsync(x, 0, sizeof(double) * ctx->n, ctx->s));
        if (!(bn == bn)) return fail(ctx, M1_ERR_NONFINITE, "non-finite right-hand side");
        return bicgstab_solve<double>(ctx, ops, b, x, o->gmres_rtol * bn, o->gmres_max, ctx->V, iters, res, conv);
    }
    return gmres64(ctx, ops, b, x, o->gmres_rtol, o->restart, o->gmres_max, iters, bnorm, res, conv);
}

m1_status m1_gmres_solve(m1_ctx* ctx, double dt, const double* U, const double* b, double* x,
                         const m1_solver_opts* opts, m1_solve_info* info, m1_mem mem) {
    if (!ctx || !b || !x) return M1_ERR_ARG;
    m1_solver_opts o;
    m1_default_opts(&o);
    if (opts) o = *opts;
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    if (U)
        CKS(copy_in(ctx, ctx->U, U, sizeof(double) * ctx->n, mem));
    else
        CK(cudaMemcpyAsync(ctx->U, ctx->Un, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s));
    CKS(copy_in(ctx, ctx->Rt, b, sizeof(double) * ctx->n, mem));
    int it = 0, ref = 0;
    double bn = 0, rs = 0;
    bool conv = false;
    CKS(linear_solve(ctx, dt, ctx->U, ctx->Rt, ctx->delta, &o, -1, &it, &ref, &bn, &rs, &conv));
    // true residual of the returned x in FP64
    jv_f64(dev64(ctx, dt), ctx->U, ctx->delta, ctx->w, ctx->s);
    launch_axpby_f64(1.0, ctx->Rt, -1.0, ctx->w, ctx->rhs, ctx->n, ctx->s);
    count(ctx, 2);
    double tr;
    CKS(norm_f64(ctx, ctx->rhs, &tr));
    CKS(copy_out(ctx, x, ctx->delta, sizeof(double) * ctx->n, mem));
    CKS(sync(ctx));
    if (info) {
        info->converged = conv;
        info->iters = it;
        info->res0 = bn;
        info->res = tr;
    }
    return conv ? M1_OK : fail(ctx, M1_ERR_NOT_CONVERGED, "GMRES did not converge");
}

// One check of the admissibility fallback at the iterate ctx->U (residual in
// ctx->R): flag the unflagged inadmissible cells (E <= 0 or |F| > cE), or, when
// there are none and Newton has not converged, the unflagged cells whose
// largest residual component is at least a tenth of the largest one; newly
// flagged inadmissible cells of U are reset to U^n. When cells were flagged, the faces of
// flagged cells get alpha = 1 and the speeds -c, +c (FP64 and FP32 copies).
static m1_status fallback_check(m1_ctx* ctx, double dt, bool converged, long long* flagged) {
    cudaStream_t s = ctx->s;
    const long long N = ctx->N;
    unsigned long long cnt = 0;
    CK(cudaMemsetAsync(ctx->fbw, 0, 2 * sizeof(unsigned long long), s));
    launch_fallback_flag(0, ctx->nu, ctx->dim, N, ctx->d.c, 0.0, ctx->U, ctx->R, ctx->Un, ctx->fb, ctx->fbw, s);
    count(ctx, 1);
    CK(cudaMemcpyAsync(ctx->hpin, ctx->fbw, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CKS(sync(ctx));
    memcpy(&cnt, ctx->hpin, sizeof(cnt));
    if (cnt == 0 && !converged) {
        launch_residual_absmax(ctx->nu, N, ctx->R, ctx->fbw + 1, s);
        count(ctx, 1);
        CK(cudaMemcpyAsync(ctx->hpin, ctx->fbw + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CKS(sync(ctx));
        unsigned long long bits = 0;
        memcpy(&bits, ctx->hpin, sizeof(bits));
        double rmax = 0.0;
        memcpy(&rmax, &bits, sizeof(rmax));
        if (rmax > 0.0) {
            launch_fallback_flag(1, ctx->nu, ctx->dim, N, ctx->d.c, 0.1 * rmax, ctx->U, ctx->R, ctx->Un, ctx->fb,
                                 ctx->fbw, s);
            count(ctx, 1);
            CK(cudaMemcpyAsync(ctx->hpin, ctx->fbw, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            CKS(sync(ctx));
            memcpy(&cnt, ctx->hpin, sizeof(cnt));
        }
    }
    *flagged = (long long)cnt;
    if (cnt > 0) {
        ctx->fb_on = true;
        TK t(ctx, M1_K_VECTOR);
        launch_fallback_faces(dev64(ctx, dt), ctx->fb, ctx->f64.lam_p, ctx->f64.lam_m, ctx->f64.alpha, s);
        for (int a = 0; a < ctx->dim; ++a) {
            launch_f64_to_f32(ctx->f64.alpha[a], ctx->f32.alpha[a], ctx->nfaces[a], s);
            launch_f64_to_f32(ctx->f64.lam_p[a], ctx->f32.lam_p[a], ctx->nfaces[a], s);
            launch_f64_to_f32(ctx->f64.lam_m[a], ctx->f32.lam_m[a], ctx->nfaces[a], s);
        }
        count(ctx, 4 * ctx->dim);
    }
    return M1_OK;
}

m1_status m1_implicit_step(m1_ctx* ctx, double dt, const m1_solver_opts* opts, m1_step_info* info) {
    if (!ctx) return M1_ERR_ARG;
    if (!(dt > 0.0)) return fail(ctx, M1_ERR_ARG, "dt must be positive");
    m1_solver_opts o;
    m1_default_opts(&o);
    if (opts) o = *opts;
    if (o.restart < 1 || o.restart > kMaxRestart) return fail(ctx, M1_ERR_ARG, "restart must be in [1, 30]");
    const bool fbk = o.realizability != 0;
    if (fbk && ctx->d.implicit_eigs && !ctx->d.fixed_eigs)
        return fail(ctx, M1_ERR_ARG, "realizability = 1 needs frozen (implicit_eigs = 0) or fixed wave speeds");
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    m1_step_info inf{};
    cudaStream_t s = ctx->s;
    // a fresh flagged set per step
    ctx->fb_on = false;
    ctx->fb_cells = 0;
    CK(cudaMemsetAsync(ctx->fb, 0, (size_t)ctx->N, s));
    CK(cudaEventRecord(ctx->ev0, s));
    // alpha and the time-n wave speeds are the first stage of every step
    CKS(refresh(ctx));
    const long long n = ctx->n;
    CK(cudaMemcpyAsync(ctx->U, ctx->Un, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double r0, rn;
    if (ctx->fp64_mode == M1_FP64_AUTO && ctx->fp64_df_ok) {
        // R(U^n) in FP64 (the reference) and in double words: their difference is
        // the double-word rounding floor at this step's magnitudes
        ctx->fp64_df = false;
        CKS(residual_norm(ctx, dev64(ctx, dt), ctx->U, ctx->R, &r0));
        Dev<double> gd = dev64(ctx, dt);
        gd.df = 1;
        double rd;
        CKS(residual_norm(ctx, gd, ctx->U, ctx->Rt, &rd));
        if (ctx->fp64_df_ok && std::isfinite(r0) && r0 > 0.0) {
            launch_axpby_f64(1.0, ctx->R, -1.0, ctx->Rt, ctx->Rt, n, s);
            count(ctx, 1);
            double d;
            CKS(norm_f64(ctx, ctx->Rt, &d));
            inf.fp64_floor = d / r0;
            ctx->fp64_df = o.newton_rtol * r0 >= 32.0 * d;
        }
    } else {
        ctx->fp64_df = ctx->fp64_df_ok;
        CKS(residual_norm(ctx, dev64(ctx, dt), ctx->U, ctx->R, &r0));
    }
    Dev<double> g = dev64(ctx, dt);
    inf.res0 = r0;
    if (!(r0 == r0) || isinf(r0)) {
        if (info) *info = inf;
        return fail(ctx, M1_ERR_NONFINITE, "non-finite initial residual");
    }
    rn = r0;
    m1_status result = M1_OK;
    int since = 0;  // Newton steps since the last admissibility check
    double rprev = 0.0, eta_prev = 0.1;  // Eisenstat-Walker forcing: the previous ||R|| and eta
    while (true) {
        const bool done = rn <= o.newton_rtol * r0;
        if (fbk && (done || (o.check_every > 0 && since >= o.check_every))) {
            since = 0;
            long long nf = 0;
            CKS(fallback_check(ctx, dt, done, &nf));
            if (nf > 0) {
                ctx->fb_cells += nf;
                inf.fallback_rounds++;
                rprev = 0.0;  // a new scheme: the forcing restarts
                g = dev64(ctx, dt);
                CKS(residual_norm(ctx, g, ctx->Un, ctx->Rt, &r0));  // the reference of the grown scheme
                CKS(residual_norm(ctx, g, ctx->U, ctx->R, &rn));
                if (!(r0 == r0) || isinf(r0) || !(rn == rn) || isinf(rn)) {
                    result = fail(ctx, M1_ERR_NONFINITE, "non-finite residual after flagging");
                    break;
                }
                continue;
            }
        }
        if (done || inf.newton_iters >= o.newton_max) break;
        // delta solves J delta = -R
        launch_axpby_f64(-1.0, ctx->R, 0.0, ctx->R, ctx->Rt, n, s);
        count(ctx, 1);
        int it = 0, ref = 0;
        double bn, rs;
        bool conv;
        m1_solver_opts ol = o;
        if (o.forcing == 1) {  // Eisenstat-Walker, choice 2
            double eta = 0.1;
            if (rprev > 0.0) {
                const double q = rn / rprev;
                eta = 0.9 * q * q;
                const double sg = 0.9 * eta_prev * eta_prev;
                if (sg > 0.1) eta = std::max(eta, sg);
            }
            eta = std::min(std::max(eta, o.gmres_rtol), 0.1);
            eta = std::max(eta, std::min(0.1, 0.5 * o.newton_rtol * r0 / rn));
            ol.gmres_rtol = eta;
            eta_prev = eta;
        }
        rprev = rn;
        m1_status ls =
            linear_solve(ctx, dt, ctx->U, ctx->Rt, ctx->delta, &ol, inf.newton_iters, &it, &ref, &bn, &rs, &conv);
        inf.gmres_iters += it;
        inf.refinements += ref;
        if (ls != M1_OK) {
            result = ls;
            break;
        }
        if (ctx->fb_on) {  // flagged cells stay admissible
            launch_admissible_theta(ctx->nu, ctx->dim, ctx->N, ctx->d.c, ctx->U, ctx->delta, ctx->fb, s);
            count(ctx, 1);
        }
        double theta = 1.0, rt = 0.0;
        for (int ls_it = 0; ls_it < 7; ++ls_it) {
            launch_axpby_f64(theta, ctx->delta, 1.0, ctx->U, ctx->Ut, n, s);
            count(ctx, 1);
            CKS(residual_norm(ctx, g, ctx->Ut, ctx->Rt, &rt));
            if (!o.line_search || rt <= (1.0 - 1e-4 * theta) * rn) break;
            theta *= 0.5;
        }
        std::swap(ctx->U, ctx->Ut);
        std::swap(ctx->R, ctx->Rt);
        rn = rt;
        if (inf.newton_iters < M1_HIST) {
            inf.res_hist[inf.newton_iters] = rn;
            inf.gmres_hist[inf.newton_iters] = it;
            inf.theta_hist[inf.newton_iters] = theta;
        }
        inf.newton_iters++;
        since++;
        ctx->st.newton_iters++;
        if (!(rn == rn) || isinf(rn)) {
            result = fail(ctx, M1_ERR_NONFINITE, "non-finite residual in Newton");
            break;
        }
    }
    inf.res0 = r0;
    inf.res = rn;
    inf.converged = (result == M1_OK) && rn <= o.newton_rtol * r0;
    inf.fp64_double_word = ctx->fp64_df ? 1 : 0;
    ctx->fp64_df = ctx->fp64_df_ok;  // outside implicit steps the mode alone decides
    inf.fallback_cells = ctx->fb_cells;
    if (ctx->fb_on) {  // the face arrays carry the fallback: recompute them before the next use
        ctx->fb_on = false;
        ctx->dirty = true;
    }
    CK(cudaMemsetAsync(ctx->viol, 0, sizeof(unsigned long long), s));
    launch_realizability(ctx->U, ctx->dim, ctx->N, ctx->d.c, ctx->viol, s);
    count(ctx, 1);
    CK(cudaMemcpyAsync(ctx->Unew, ctx->U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (inf.converged && o.advance) {
        CK(cudaMemcpyAsync(ctx->Un, ctx->U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        ctx->dirty = true;
    }
    CK(cudaEventRecord(ctx->ev1, s));
    unsigned long long hv = 0;
    CK(cudaMemcpyAsync(ctx->hpin, ctx->viol, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CKS(sync(ctx));
    memcpy(&hv, ctx->hpin, sizeof(hv));
    inf.realizability_violations = (long long)hv;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    inf.time_ms = ms;
    ctx->st.implicit_steps++;
    if (info) *info = inf;
    if (ctx->dirty) CKS(prepare(ctx));
    if (result != M1_OK) return result;
    if (!inf.converged) return fail(ctx, M1_ERR_NOT_CONVERGED, "Newton did not converge");
    return M1_OK;
}

m1_status m1_get_fallback(const m1_ctx* cctx, unsigned char* mask, m1_mem mem) {
    m1_ctx* ctx = const_cast<m1_ctx*>(cctx);
    if (!ctx || !mask) return M1_ERR_ARG;
    if (!ctx->fb) {
        if (mem == M1_MEM_DEVICE)
            CK(cudaMemsetAsync(mask, 0, (size_t)ctx->N, ctx->s));
        else
            memset(mask, 0, (size_t)ctx->N);
        return sync(ctx);
    }
    CKS(copy_out(ctx, mask, ctx->fb, (size_t)ctx->N, mem));
    return sync(ctx);
}

m1_status m1_set_preconditioner(m1_ctx* ctx, m1_nn* nn) {
    if (!ctx) return M1_ERR_ARG;
    if (!nn) {
        ctx->nn = nullptr;
        return M1_OK;
    }
    if (ctx->dim != 2 || ctx->d.gas_coupling)
        return fail(ctx, M1_ERR_ARG, "the learned preconditioner is 2D radiation-only");
    if (nn_height(nn) != ctx->d.n[1] || nn_width(nn) != ctx->d.n[0])
        return fail(ctx, M1_ERR_ARG, "network size differs from the grid (build it for n[1] x n[0], batch 1)");
    CKS(dalloc(ctx, &ctx->logsig, ctx->N));
    CKS(dalloc(ctx, &ctx->nn_static, 4 * ctx->N));
    CKS(dalloc(ctx, &ctx->nn_null, 3 * ctx->N));
    ctx->nn = nn;
    ctx->dirty = true;
    return M1_OK;
}

m1_status m1_set_learned_form(m1_ctx* ctx, int form) {
    if (!ctx) return M1_ERR_ARG;
    if (form != M1_LEARNED_ADDITIVE && form != M1_LEARNED_TWO_STAGE && form != M1_LEARNED_TWO_STAGE_ALL)
        return fail(ctx, M1_ERR_ARG, "unknown learned-preconditioner form");
    ctx->nn_form = form;
    return M1_OK;
}

m1_status m1_nn_make_pair(m1_ctx* ctx, double dt, const double* U, const double* e, float* x, float* t,
                          m1_mem mem) {
    if (!ctx || !e || !x || !t) return M1_ERR_ARG;
    if (ctx->dim != 2 || ctx->d.gas_coupling) return fail(ctx, M1_ERR_ARG, "pairs are 2D radiation-only");
    CKS(dalloc(ctx, &ctx->logsig, ctx->N));
    CKS(dalloc(ctx, &ctx->nn_static, 4 * ctx->N));
    CKS(prepare(ctx));
    CKS(ensure_work(ctx));
    launch_logsig(ctx->sig_f, ctx->N, (ctx->d.hi[0] - ctx->d.lo[0]) / ctx->d.n[0], ctx->logsig, ctx->s);
    if (U)
        CKS(copy_in(ctx, ctx->U, U, sizeof(double) * ctx->n, mem));
    else
        CK(cudaMemcpyAsync(ctx->U, ctx->Un, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s));
    CKS(copy_in(ctx, ctx->delta, e, sizeof(double) * ctx->n, mem));
    Dev<double> g = dev64(ctx, dt);
    jv_f64(g, ctx->U, ctx->delta, ctx->w, ctx->s);  // r = J e
    CKS(build_precond(ctx, g, ctx->U));
    launch_bj_apply_f64(ctx->nu, ctx->N, ctx->binv, ctx->w, ctx->z, ctx->s);  // J_bj^-1 r
    launch_axpby_f64(1.0, ctx->delta, -1.0, ctx->z, ctx->tmp, ctx->n, ctx->s);  // e - J_bj^-1 r
    count(ctx, 4);
    double rn;
    CKS(norm_f64(ctx, ctx->w, &rn));
    const double scale = rn > 0.0 ? rn / sqrt((double)ctx->n) : 1.0;
    float* xd = nullptr;
    float* td = nullptr;
    if (mem == M1_MEM_DEVICE) {
        xd = x;
        td = t;
    } else {
        CKS(dalloc(ctx, &ctx->pair_x, 7 * ctx->N));
        CKS(dalloc(ctx, &ctx->pair_t, 3 * ctx->N));
        xd = ctx->pair_x;
        td = ctx->pair_t;
    }
    launch_nn_static_f64(ctx->U, ctx->N, ctx->d.c, ctx->logsig, ctx->nn_static, ctx->s);
    launch_pack_pair(ctx->w, ctx->tmp, ctx->N, ctx->nn_static, scale, xd, td, ctx->s);
    count(ctx, 2);
    if (mem != M1_MEM_DEVICE) {
        CK(cudaMemcpyAsync(x, xd, sizeof(float) * 7 * ctx->N, cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaMemcpyAsync(t, td, sizeof(float) * 3 * ctx->N, cudaMemcpyDeviceToHost, ctx->s));
    }
    return sync(ctx);
}

m1_status m1_set_fp64_arithmetic(m1_ctx* ctx, int mode) {
    if (!ctx) return M1_ERR_ARG;
    if (mode != M1_FP64_AUTO && mode != M1_FP64_NATIVE && mode != M1_FP64_DOUBLE_WORD)
        return fail(ctx, M1_ERR_ARG, "unknown FP64 arithmetic mode");
    ctx->fp64_mode = mode;
    ctx->fp64_df = ctx->fp64_df_ok = mode == M1_FP64_DOUBLE_WORD || (mode == M1_FP64_AUTO && fp64_auto_df(ctx->d));
    return M1_OK;
}

m1_status m1_get_fp64_arithmetic(const m1_ctx* ctx, int* mode, long long* fallbacks) {
    if (!ctx) return M1_ERR_ARG;
    if (mode) *mode = ctx->fp64_df ? M1_FP64_DOUBLE_WORD : M1_FP64_NATIVE;
    if (fallbacks) *fallbacks = ctx->fp64_df_fallbacks;
    return M1_OK;
}

m1_status m1_profile(m1_ctx* ctx, int enable) {
    if (!ctx) return M1_ERR_ARG;
    CKS(sync(ctx));
    if (enable && ctx->evs.empty()) {
        const int pairs = 2048;
        ctx->evs.resize(2 * pairs);
        ctx->ev_cls.resize(pairs);
        for (auto& e : ctx->evs) CK(cudaEventCreate(&e));
    }
    ctx->prof = enable != 0;
    ctx->ev_used = 0;
    for (int k = 0; k < M1_K_CLASSES; ++k) {
        ctx->st.kernel_ms[k] = 0.0;
        ctx->st.kernel_count[k] = 0;
    }
    return M1_OK;
}

m1_status m1_stats(const m1_ctx* ctx, m1_stats_t* out) {
    if (!ctx || !out) return M1_ERR_ARG;
    *out = ctx->st;
    return M1_OK;
}

const char* m1_last_error(const m1_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"
