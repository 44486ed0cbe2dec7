// m1_noalloc.cu — allocation-free residual (m1_residual_noalloc in m1.h).
//
// For callers that cannot allocate device memory at the call site. The
// working memory that m1_residual keeps in its context (the time-n face data
// lambda+-, alpha, and the per-block partial sums of ||R||^2) lives here in one
// file-scope __device__ array sized for M1_NOALLOC_MAX_CELLS cells. The same
// kernels as the context path run on it, so the results are the same.
//
// The array's device address is looked up with cudaGetSymbolAddress once per
// CUDA context, at the first call made while that context is current, and
// cached under the context's unique id (cuCtxGetId; ids are never reused within
// a process). A device reset or a re-created primary context therefore gets a
// fresh lookup instead of a stale address. Host code never passes the array's
// host-side name to a kernel. Calls share the array: every
// entry is written before it is read within a call, nothing accumulates across
// calls, and calls that overlap on the GPU race.
#include <cuda.h>

#include <mutex>

#include "../../include/m1.h"
#include "m1_internal.h"

namespace {

constexpr long long kMaxCells = M1_NOALLOC_MAX_CELLS;
// per axis at most 2N faces, three face arrays (lambda+, lambda-, alpha), three axes
constexpr long long kFaceDoubles = 3LL * 3LL * 2LL * kMaxCells;
constexpr long long kPartials = (kMaxCells + 255) / 256;
constexpr long long kScratchDoubles = kFaceDoubles + kPartials + 64;

}  // namespace

// the working array: one per GPU that loads the library, zero at load time
static __device__ __align__(256) double m1_noalloc_scratch[kScratchDoubles];

namespace {

// (context id, device address) pairs; a full table overwrites its oldest entry
constexpr int kCacheSlots = 64;
struct ScratchSlot {
    unsigned long long ctx_id;
    void* addr;
};
ScratchSlot g_slots[kCacheSlots] = {};
int g_next_slot = 0;
std::mutex g_scratch_mu;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// the unique id of the CUDA context current on this thread (the runtime makes
// the device's primary context current first)
m1_status current_context_id(unsigned long long* id) {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return M1_ERR_CUDA;
        get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
        get_id = reinterpret_cast<PfnCtxGetId>(f2);
    }
    // cudaSetDevice makes the device's primary context current on this thread
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return M1_ERR_CUDA;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return M1_ERR_CUDA;
    return get_id(ctx, id) == CUDA_SUCCESS ? M1_OK : M1_ERR_CUDA;
}

m1_status scratch_address(double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = 0;
    const m1_status st = current_context_id(&id);
    if (st != M1_OK) return st;
    for (const ScratchSlot& e : g_slots)
        if (e.addr && e.ctx_id == id) {
            *out = static_cast<double*>(e.addr);
            return M1_OK;
        }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, m1_noalloc_scratch) != cudaSuccess || !p) return M1_ERR_CUDA;
    g_slots[g_next_slot] = ScratchSlot{id, p};
    g_next_slot = (g_next_slot + 1) % kCacheSlots;
    *out = static_cast<double*>(p);
    return M1_OK;
}

bool valid(const m1_grid_desc* d) {
    if (!d || d->dim < 1 || d->dim > 3) return false;
    for (int a = 0; a < 3; ++a) {
        if (d->n[a] < 1 || (a >= d->dim && d->n[a] != 1)) return false;
        if (a < d->dim) {
            if (!(d->hi[a] > d->lo[a])) return false;
            for (int s = 0; s < 2; ++s)
                if (d->bc[a][s] < 0 || d->bc[a][s] > 3) return false;
            if ((d->bc[a][0] == M1_BC_PERIODIC) != (d->bc[a][1] == M1_BC_PERIODIC)) return false;
        }
    }
    return d->c > 0.0 && d->a_r > 0.0 && d->lambda_floor >= 0.0;
}

}  // namespace

extern "C" m1_status m1_residual_noalloc(const m1_grid_desc* d, double dt, const m1_device_fields* f,
                                         const double* U, double* R, double* norm2, void* cuda_stream) {
    using namespace m1;
    if (!valid(d) || !f || !U || !R || !f->Un || !f->sigma_a) return M1_ERR_ARG;
    if (d->gas_coupling && !f->rho_cv) return M1_ERR_ARG;
    const long long N = (long long)d->n[0] * d->n[1] * d->n[2];
    if (N > kMaxCells) return M1_ERR_ARG;  // larger than the static working array
    for (int a = 0; a < d->dim; ++a)
        for (int s = 0; s < 2; ++s)
            if (d->bc[a][s] == M1_BC_DIRICHLET && (!f->bE[a][s] || !f->bF[a][s])) return M1_ERR_ARG;
    double* base = nullptr;
    const m1_status st = scratch_address(&base);
    if (st != M1_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    Dev<double> g{};
    g.dim = d->dim;
    g.nx = d->n[0];
    g.ny = d->n[1];
    g.nz = d->n[2];
    g.N = N;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = d->n[a];
        const double dx = (d->hi[a] - d->lo[a]) / d->n[a];
        g.dx[a] = dx;
        g.inv_dx[a] = 1.0 / dx;
        g.bM[a] = N / d->n[a];
        for (int sd = 0; sd < 2; ++sd) {
            g.bc[a][sd] = d->bc[a][sd];
            g.bE[a][sd] = f->bE[a][sd];
            g.bF[a][sd] = f->bF[a][sd];
            g.bmask[a][sd] = f->bmask[a][sd];
        }
    }
    g.stride[0] = 1;
    g.stride[1] = d->n[0];
    g.stride[2] = (long long)d->n[0] * d->n[1];
    g.c = d->c;
    g.a_r = d->a_r;
    g.dt = dt;
    g.lambda_floor = d->lambda_floor;
    g.gas = d->gas_coupling;
    g.wb = d->well_balanced;
    g.ap = d->ap_correction;
    g.fixed_eigs = d->fixed_eigs;
    g.wb_boundary = d->wb_boundary;
    g.implicit_eigs = d->implicit_eigs;
    g.sig_a = f->sigma_a;
    g.sig_f = f->sigma_f ? f->sigma_f : f->sigma_a;
    g.B = d->gas_coupling ? nullptr : f->B;
    g.S = f->S;
    g.rho_cv = f->rho_cv;
    g.Un = f->Un;

    // carve the working array: face data per axis, then the partials, then ||R||^2
    double* lam_p[3] = {nullptr, nullptr, nullptr};
    double* lam_m[3] = {nullptr, nullptr, nullptr};
    double* alpha[3] = {nullptr, nullptr, nullptr};
    double* p = base;
    for (int a = 0; a < d->dim; ++a) {
        const long long nf = N / d->n[a] * (d->n[a] + 1);
        lam_p[a] = p;
        lam_m[a] = p + nf;
        alpha[a] = p + 2 * nf;
        p += 3 * nf;
        g.lam_p[a] = lam_p[a];
        g.lam_m[a] = lam_m[a];
        g.alpha[a] = alpha[a];
    }
    double* partials = base + kFaceDoubles;
    double* nrm = partials + kPartials;

    launch_faces_time_n(g, lam_p, lam_m, alpha, s);
    const int nb = launch_residual_f64(g, U, R, partials, kPartials, s);
    launch_finish_sum(partials, nb, 1, nrm, s);
    if (norm2 && cudaMemcpyAsync(norm2, nrm, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return M1_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? M1_OK : M1_ERR_CUDA;
}
