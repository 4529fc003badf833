// Host orchestration of the multigrid-preconditioned MINRES solve (Section 5): hierarchy set-up,
// the V-cycle, the Lanczos estimate of the Jacobi weights, MINRES, and the mixed-precision
// iterative refinement. Every step runs in the kernels of apply.cu, mg.cu and krylov.cu; the host
// only sequences launches and reads back scalars.
#include <chrono>
#include <cmath>
#include <limits>

#include "pbm_internal.h"

namespace pbm {

void mr_scalars(pbm_grid* g, cudaStream_t st);
void mr_init(pbm_grid* g, cudaStream_t st);
void add_f32(double* x, const float* d, int64_t n, cudaStream_t st, double sign);
void mr_lanczos2(pbm_grid* g, bool fp32, const void* Az, void* v0, void* v1, int64_t n, cudaStream_t st);
void mr_update2(pbm_grid* g, bool fp32, void* zc, const void* zn, void* d1, void* d2, void* x, int64_t n,
                cudaStream_t st);
void cast_dot(pbm_grid* g, const float* src, double* dst, const double* other, int64_t n, int slot, cudaStream_t st);
void lz_start(pbm_grid* g, double* v, double* t, double* vprev, const double* diag, int64_t n, cudaStream_t st);
void lz_b(pbm_grid* g, double* w, const double* v, const double* vprev, const double* sdiag, int64_t n, int j0,
          int j, int rset, cudaStream_t st);
void lz_next(pbm_grid* g, const double* w, double* v, double* vprev, double* t, const double* diag, int64_t n, int j,
             cudaStream_t st);

// ------------------------------------------------------------------------------------------------
// operator application on level k
// ------------------------------------------------------------------------------------------------
void level_apply(pbm_grid* g, int k, bool fp32, bool op_s, const ApplyArgs& a0, cudaStream_t st) {
    ApplyArgs a = a0;
    a.with_alpha = op_s;
    if (k == 0) {
        const void* w = op_s ? (fp32 ? (const void*)g->w32 : (const void*)g->w64)
                             : (fp32 ? (const void*)g->rho32 : (const void*)g->rho);
        if (op_s)
            launch_fine(g, fp32, w, fp32 ? (const void*)g->d32 : (const void*)g->d64,
                        fp32 ? (const void*)g->u32 : (const void*)g->u64, a, st);
        else
            launch_fine(g, fp32, w, nullptr, nullptr, a, st);
    } else {
        launch_coarse(g, k, fp32, a, st);
    }
}

static ApplyArgs args(const void* x, void* y, int mode, const void* b = nullptr, const void* diag = nullptr,
                      const double* om = nullptr, int slot = -1) {
    ApplyArgs a{};
    a.x = x;
    a.y = y;
    a.b = b;
    a.diag = diag;
    a.omega = om;
    a.mode = mode;
    a.dot_slot = slot;
    return a;
}

static size_t esz(bool fp32) { return fp32 ? sizeof(float) : sizeof(double); }

void vcycle(pbm_grid* g, int k, bool fp32, bool op_s, const void* b, void* x, int dot_slot, cudaStream_t st,
            bool first_done);

// V-cycle with multicolour Gauss-Seidel smoothing: every sweep is one operator launch per colour (24 dof
// colours, and alpha last for S) with the EPI_GS0 + c epilogue, forward before the coarse correction and
// backward after it; pre-smoothing starts from x = 0 (no sweep is fused into the restriction)
static void vcycle_gs(pbm_grid* g, int k, bool fp32, bool op_s, const void* b, void* x, int dot_slot,
                      cudaStream_t st) {
    Level& L = g->L[k];
    const int64_t nv = L.g.n() + (op_s ? 1 : 0);
    const size_t es = fp32 ? sizeof(float) : sizeof(double);
    void* t = fp32 ? (void*)L.t32 : (void*)L.t64;
    void* r = fp32 ? (void*)L.r32 : (void*)L.r64;
    const void* D = fp32 ? (const void*)L.idiag32 : (const void*)L.idiag64;
    const int ncol = op_s ? kGsColours + 1 : kGsColours;
    const int pre = g->desc.pre_sweeps, post = g->desc.post_sweeps;
    vec_zero(x, nv * es, st);
    void* cur = x;
    void* oth = t;
    for (int sw = 0; sw < pre; ++sw)
        for (int c = 0; c < ncol; ++c) {
            level_apply(g, k, fp32, op_s, args(cur, oth, EPI_GS0 + c, b, D), st);
            std::swap(cur, oth);
        }
    if (cur != x) PBM_CUDA(cudaMemcpyAsync(x, cur, nv * es, cudaMemcpyDeviceToDevice, st));
    level_apply(g, k, fp32, op_s, args(x, r, EPI_RESID, b), st);
    Level& C = g->L[k + 1];
    void* bc = fp32 ? (void*)C.b32 : (void*)C.b64;
    void* xc = fp32 ? (void*)C.x32 : (void*)C.x64;
    launch_restrict(g, k, fp32, r, bc, op_s, 1.0, st, nullptr);
    vcycle(g, k + 1, fp32, op_s, bc, xc, -1, st, false);
    launch_prolong_add(g, k, fp32, xc, x, op_s, st);
    cur = x;
    oth = t;
    for (int sw = 0; sw < post; ++sw)
        for (int c = ncol - 1; c >= 0; --c) {
            const bool last = sw == post - 1 && c == 0;
            level_apply(g, k, fp32, op_s, args(cur, oth, EPI_GS0 + c, b, D, nullptr, last ? dot_slot : -1), st);
            std::swap(cur, oth);
        }
    if (cur != x) PBM_CUDA(cudaMemcpyAsync(x, cur, nv * es, cudaMemcpyDeviceToDevice, st));
    if (post == 0 && dot_slot >= 0) launch_dot(g, fp32, x, b, nv, dot_slot, st);
}

// ------------------------------------------------------------------------------------------------
// V-cycle: x = M^{-1} b on level k (x overwritten). If dot_slot >= 0, red[dot_slot] = x . b.
// ------------------------------------------------------------------------------------------------
// first_done: the caller already wrote the first pre-smoothing sweep omega D^{-1} b into the buffer
// the sweep sequence starts from (x for an odd number of pre-sweeps, else the level's t)
void vcycle(pbm_grid* g, int k, bool fp32, bool op_s, const void* b, void* x, int dot_slot, cudaStream_t st,
            bool first_done = false) {
    Level& L = g->L[k];
    const int64_t nv = L.g.n() + (op_s ? 1 : 0);
    if (k == g->levels - 1) {
        launch_coarsest_solve(g, fp32, b, x, op_s, st);
        if (dot_slot >= 0) launch_dot(g, fp32, x, b, nv, dot_slot, st);
        return;
    }
    void* t = fp32 ? (void*)L.t32 : (void*)L.t64;
    void* r = fp32 ? (void*)L.r32 : (void*)L.r64;
    const void* D = fp32 ? (const void*)L.idiag32 : (const void*)L.idiag64;
    const double* om = &g->sc->mr[16 + k];
    if (g->desc.smoother == PBM_SMOOTHER_GAUSS_SEIDEL) {
        vcycle_gs(g, k, fp32, op_s, b, x, dot_slot, st);
        return;
    }
    const int pre = g->desc.pre_sweeps, post = g->desc.post_sweeps;
    // pre-smoothing from x = 0: the first sweep is x = omega D^-1 b; arrange the ping-pong so that
    // the last pre-sweep lands in x
    void* cur = (pre % 2 == 1) ? x : t;
    void* oth = (cur == x) ? t : x;
    // Chebyshev: step s >= 1 of a pass is EPI_CHEB with that step's coefficients; its previous iterate
    // is the other ping-pong buffer (zero before the pre-smoothing's second step: c1 = 0 there)
    const bool cheb = g->desc.smoother == PBM_SMOOTHER_CHEBYSHEV;
    auto step_mode = [&](int s) { return (cheb && s >= 1) ? EPI_CHEB : EPI_JACOBI; };
    auto step_coef = [&](int s, bool pre_pass) {
        return (cheb && s >= 1) ? &g->sc->cheb[k][cheb_slot(s, pre_pass && s == 1)] : om;
    };
    if (pre >= 1) {
        if (!first_done) launch_scale_diag_first(g, k, fp32, b, cur, op_s, st);
        for (int s = 1; s < pre; ++s) {
            level_apply(g, k, fp32, op_s, args(cur, oth, step_mode(s), b, D, step_coef(s, true)), st);
            std::swap(cur, oth);
        }
    } else {
        vec_zero(x, nv * esz(fp32), st);
        cur = x;
        oth = t;
    }
    // residual, restriction, coarse correction, prolongation
    level_apply(g, k, fp32, op_s, args(x, r, EPI_RESID, b), st);
    Level& C = g->L[k + 1];
    void* bc = fp32 ? (void*)C.b32 : (void*)C.b64;
    void* xc = fp32 ? (void*)C.x32 : (void*)C.x64;
    // the restriction also writes the coarse level's first smoothing sweep, unless that level is the
    // coarsest (exact solve)
    const bool fuse = (k + 1 < g->levels - 1) && pre >= 1;
    void* xfirst = nullptr;
    if (fuse) xfirst = (pre % 2 == 1) ? xc : (fp32 ? (void*)C.t32 : (void*)C.t64);
    launch_restrict(g, k, fp32, r, bc, op_s, 1.0, st, xfirst);
    vcycle(g, k + 1, fp32, op_s, bc, xc, -1, st, fuse);
    launch_prolong_add(g, k, fp32, xc, x, op_s, st);
    // post-smoothing
    cur = x;
    oth = t;
    for (int s = 0; s < post; ++s) {
        const bool last = (s == post - 1);
        level_apply(g, k, fp32, op_s, args(cur, oth, step_mode(s), b, D, step_coef(s, false), last ? dot_slot : -1),
                    st);
        std::swap(cur, oth);
    }
    if (cur != x) PBM_CUDA(cudaMemcpyAsync(x, cur, nv * esz(fp32), cudaMemcpyDeviceToDevice, st));
    if (post == 0 && dot_slot >= 0) launch_dot(g, fp32, x, b, nv, dot_slot, st);
}

// ------------------------------------------------------------------------------------------------
// largest eigenvalue of a symmetric tridiagonal matrix (bisection on the Sturm count)
// ------------------------------------------------------------------------------------------------
static double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
    const int k = int(a.size());
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto count_below = [&](double x) {  // eigenvalues < x
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < k; ++i) {
            const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
            d = a[i] - x - (i > 0 ? bb / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(mid) >= k) hi = mid;
        else lo = mid;
    }
    return hi;
}

// Lanczos estimate of lambda_max(D^{-1} A) on level k, enqueued on `st` with reduction set `rset`:
// the coefficients go to sc->lz_a / lz_b from index k * steps; lanczos_finish reads them on the host.
// Every level has its own vectors (its V-cycle work vectors), reduction slot and set, so the levels
// can run on concurrent streams.
static void lanczos_issue(pbm_grid* g, int k, bool op_s, int rset, cudaStream_t st) {
    Level& L = g->L[k];
    const int64_t nv = L.g.n() + (op_s ? 1 : 0);
    double* v = L.x64;
    double* vp = L.b64;
    double* t = L.r64;
    double* w = L.t64;
    const int steps = g->desc.lanczos_steps;
    const int j0 = k * steps;
    launch_inverse_sqrt(L.diag64, L.sdiag64, nv, st);
    lz_start(g, v, t, vp, L.sdiag64, nv, st);
    // a_j = (A t) . t with t = D^{-1/2} v is the operator launch's fused dot product. Mixed grids
    // apply the FP32 operators the smoother will use (the weight is an estimate; the Lanczos
    // vectors and scalars stay FP64); FP64 grids the FP64 ones.
    const bool op32 = g->desc.precision == PBM_MIXED;
    float* t32 = op32 ? L.x32 : nullptr;
    float* w32 = op32 ? L.t32 : nullptr;
    const int slot = 40 + k;
    for (int j = 0; j < steps; ++j) {
        ApplyArgs a = args(op32 ? (const void*)t32 : (const void*)t, op32 ? (void*)w32 : (void*)w, EPI_APPLY, nullptr,
                           nullptr, nullptr, slot);
        a.rset = rset;
        if (op32) {
            launch_cast(t, false, t32, true, nv, st);
            level_apply(g, k, true, op_s, a, st);
            launch_cast(w32, true, w, false, nv, st);
        } else {
            level_apply(g, k, false, op_s, a, st);
        }
        PBM_CUDA(cudaMemcpyAsync(&g->sc->lz_a[j0 + j], &g->sc->red[slot], sizeof(double), cudaMemcpyDeviceToDevice,
                                 st));
        lz_b(g, w, v, vp, L.sdiag64, nv, j0, j, rset, st);
        lz_next(g, w, v, vp, t, L.sdiag64, nv, j0 + j, st);
    }
}

// host side, after the coefficients of level k are in sc_host: the largest Ritz value and the weight
static void lanczos_finish(pbm_grid* g, int k) {
    Level& L = g->L[k];
    const int steps = g->desc.lanczos_steps;
    const int j0 = k * steps;
    std::vector<double> a, b;
    for (int j = 0; j < steps; ++j) {
        a.push_back(g->sc_host->lz_a[j0 + j]);
        const double bj = g->sc_host->lz_b[j0 + j];
        if (!(bj > 0.0) || j == steps - 1) break;
        b.push_back(bj);
    }
    b.resize(a.size() > 0 ? a.size() - 1 : 0);
    L.lambda_max = tridiag_max_eig(a, b);
    if (!(L.lambda_max > 0.0) || !std::isfinite(L.lambda_max)) fail(PBM_ENONFINITE, "Lanczos estimate is not positive");
    if (g->desc.smoother == PBM_SMOOTHER_CHEBYSHEV) {
        // Chebyshev acceleration on [lo, hi] = [0.1, 1.4] lambda: centre theta, half width delta (every
        // eigenvalue of D^-1 A up to lo + hi = 1.5 lambda is damped, so the estimate from below may be off by a
        // third, as the Jacobi weight's 2 / theta = 1.67 allows); the first
        // step of a pass is a Jacobi step with weight 1 / theta, step s >= 1 takes
        // x_{s+1} = x_s + a_s (x_s - x_{s-1}) + b_s D^-1 (b - A x_s) with rho_0 = delta / theta,
        // rho_s = 1 / (2 theta / delta - rho_{s-1}), a_s = rho_s rho_{s-1}, b_s = 2 rho_s / delta
        const double lo = 0.1 * L.lambda_max, hi = 1.4 * L.lambda_max;
        const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
        L.omega = 1.0 / theta;
        double rho = 1.0 / sigma;
        double* c = g->sc_host->cheb[k];
        for (int st = 1; st <= kChebMaxStep; ++st) {
            const double rn = 1.0 / (2.0 * sigma - rho);
            const double as = rn * rho, bs = 2.0 * rn / delta;
            for (int z = 0; z < 2; ++z) {
                double* e = c + cheb_slot(st, z == 1);
                e[0] = 1.0 + as;
                e[1] = z == 1 ? 0.0 : as;
                e[2] = bs;
                e[3] = 0.0;
            }
            rho = rn;
        }
    } else {
        L.omega = g->desc.jacobi_theta / L.lambda_max;
    }
}

static void upload_omegas(pbm_grid* g, cudaStream_t st) {
    for (int k = 0; k < g->levels; ++k) g->sc_host->mr[16 + k] = g->L[k].omega;
    PBM_CUDA(cudaMemcpyAsync(&g->sc->mr[16], &g->sc_host->mr[16], sizeof(double) * 16, cudaMemcpyHostToDevice, st));
    if (g->desc.smoother == PBM_SMOOTHER_CHEBYSHEV)
        PBM_CUDA(cudaMemcpyAsync(&g->sc->cheb[0][0], &g->sc_host->cheb[0][0], sizeof(g->sc_host->cheb),
                                 cudaMemcpyHostToDevice, st));
}

// ------------------------------------------------------------------------------------------------
// hierarchy set-up for K(w64) (op_s = false) or S (op_s = true; coefficients already in place)
// ------------------------------------------------------------------------------------------------
void setup_hierarchy(pbm_grid* g, bool op_s, cudaStream_t st) {
    const bool mixed = g->desc.precision == PBM_MIXED;
    const int nl = g->levels;
    Level& F = g->L[0];
    const int steps = g->desc.lanczos_steps;
    if (steps * std::max(1, nl - 1) > 128) fail(PBM_EINVAL, "lanczos_steps x levels exceeds 128");
    if (nl > 16) fail(PBM_EINVAL, "more than 16 levels");
    for (int i = 0; i < 19; ++i) {
        if (i < 16 && !g->side[i]) PBM_CUDA(cudaStreamCreateWithFlags(&g->side[i], cudaStreamNonBlocking));
        if (!g->side_ev[i]) PBM_CUDA(cudaEventCreateWithFlags(&g->side_ev[i], cudaEventDisableTiming));
    }
    // The Galerkin chain of the coarse levels needs only the element weights (and, for S, the table
    // of P_c^T K_e u_e), so it starts at once on side[1], beside the rest of the fine level's data on
    // `st`: the alpha border b_0 = -sum_i d_i K_i u (the chain waits for it before restricting it), the
    // W_e table of the S pass and the Jacobi diagonal. Mixed grids build the chain in FP32 from the
    // FP32 copies of the weights and u (made first): it only feeds the FP32 V-cycle, and the FP64
    // matrices are built when a call reads them (ensure_coarse64).
    if (mixed) {
        if (op_s) {
            launch_cast(g->w64, false, g->w32, true, F.g.m(), st);
            launch_cast(g->d64, false, g->d32, true, F.g.m(), st);
            launch_cast(g->u64, false, g->u32, true, F.g.n(), st);
        } else {
            launch_cast(g->rho, false, g->rho32, true, F.g.m(), st);
        }
    }
    g->coarse64_ready = !mixed;
    cudaEvent_t fork = g->side_ev[16], chain = g->side_ev[17], border = g->side_ev[18];
    PBM_CUDA(cudaEventRecord(fork, st));
    const cudaStream_t sg = g->side[1];
    if (nl >= 2) {
        PBM_CUDA(cudaStreamWaitEvent(sg, fork, 0));
        if (op_s) launch_build_what(g, sg, mixed);
        launch_build_level1(g, op_s, sg, mixed);
    }
    if (op_s) {
        launch_fine(g, false, g->d64, nullptr, nullptr, args(g->u64, F.bord64, EPI_APPLY), st);
        PBM_CUDA(cudaEventRecord(border, st));
        launch_what_hat(g, st);
    }
    launch_diag(g, 0, op_s, st);
    // From here three kinds of work overlap: the fine level's Lanczos estimate on `st`; the Galerkin
    // chain of the coarse levels on side[1], followed there by level 1's Lanczos; once the chain is
    // done, the coarsest factorisation on side[0] and the Lanczos of levels 2 .. nl - 2 on side[k].
    // Each stream has its own reduction set, vectors and slots; one synchronisation reads everything.
    if (nl >= 2) {
        if (op_s) {
            PBM_CUDA(cudaStreamWaitEvent(sg, border, 0));
            launch_restrict(g, 0, false, F.bord64, g->L[1].bord64, false, -1.0, sg);
        }
        for (int k = 1; k + 1 < nl; ++k) {
            launch_build_coarser(g, k, sg, mixed);
            if (op_s) launch_restrict(g, k, false, g->L[k].bord64, g->L[k + 1].bord64, false, 1.0, sg);
        }
        for (int k = 1; k < nl; ++k) launch_diag(g, k, op_s, sg, 1, mixed);
        if (mixed) {
            for (int k = 1; k < nl; ++k) launch_coarse_to_f32(g, k, sg, false);
            launch_coarse_to_f64(g, nl - 1, sg);   // the coarsest level's FP64 factorisation
        }
        PBM_CUDA(cudaEventRecord(chain, sg));
        PBM_CUDA(cudaStreamWaitEvent(g->side[0], chain, 0));
        build_coarsest(g, op_s, g->side[0]);
        PBM_CUDA(cudaEventRecord(g->side_ev[0], g->side[0]));
        for (int k = 1; k + 1 < nl; ++k) {
            if (k > 1) PBM_CUDA(cudaStreamWaitEvent(g->side[k], chain, 0));
            lanczos_issue(g, k, op_s, k, g->side[k]);
            PBM_CUDA(cudaEventRecord(g->side_ev[k], g->side[k]));
        }
        lanczos_issue(g, 0, op_s, 0, st);
        for (int k = 0; k + 1 < nl; ++k) PBM_CUDA(cudaStreamWaitEvent(st, g->side_ev[k], 0));
        if (nl == 2) PBM_CUDA(cudaStreamWaitEvent(st, chain, 0));
    }
    PBM_CUDA(cudaMemcpyAsync(g->sc_host->lz_a, g->sc->lz_a, sizeof(double) * steps * std::max(1, nl - 1),
                             cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaMemcpyAsync(g->sc_host->lz_b, g->sc->lz_b, sizeof(double) * steps * std::max(1, nl - 1),
                             cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaMemcpyAsync(g->sc_host->flags, g->sc->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k + 1 < nl; ++k) lanczos_finish(g, k);
    upload_omegas(g, st);
    if (nl >= 2 && g->sc_host->flags[0] != 0) fail(PBM_ENONFINITE, "coarsest matrix is not positive definite");
    g->op_ready = op_s ? 2 : 1;
}

// ------------------------------------------------------------------------------------------------
// MINRES (x holds the initial guess); returns status
//
// Vectors in the precision `fp32` (FP32 only for the inner solves of the mixed path), scalars in
// FP64 on the device. With pc32 (FP64 vectors only) the preconditioner is the FP32 V-cycle: the
// Lanczos vector is rounded to FP32, cycled, and widened back with the dot product fused.
// When the recurrence's residual estimate reaches the target the true residual is computed
// (check_true); if it is above rtol the target is tightened and the iteration continues, unless
// the true residual has not halved since the previous check (stagnation: returns PBM_ENOTCONV
// with the current iterate, which the caller may restart from).
// ------------------------------------------------------------------------------------------------
struct MrResult {
    int status = PBM_OK;
    int iters = 0;
    double relres = 0.0;
};

static void precondition(pbm_grid* g, bool fp32, bool pc32, bool op_s, const void* v, void* z, int64_t nv,
                         cudaStream_t st) {
    if (!pc32) {
        vcycle(g, 0, fp32, op_s, v, z, 1, st);
        return;
    }
    Level& F = g->L[0];
    launch_cast(v, false, F.b32, true, nv, st);
    vcycle(g, 0, true, op_s, F.b32, F.x32, -1, st);
    cast_dot(g, F.x32, (double*)z, (const double*)v, nv, 1, st);
}

// ---- MINRES loop control on the device (graph mode) ----------------------------------------------
// ctl[0] target on the residual estimate, ctl[1] iteration budget, ctl[2] iterations done,
// ctl[3] exit reason: 1 breakdown, 2 lucky (beta = 0 or r = 0), 3 estimate below target, 4 budget
__global__ void k_mr_ctl(double* ctl, double target, double budget) {
    pdl_wait();
    ctl[0] = target;
    ctl[1] = budget;
    ctl[2] = 0.0;
    ctl[3] = 0.0;
}

__device__ __forceinline__ int mr_exit_reason(const double* mr, double target, double it, double budget) {
    if (mr[13] == 1.0) return 1;
    if (mr[13] == 2.0 || mr[1] == 0.0) return 2;
    if (fabs(mr[6]) <= target * mr[7]) return 3;
    if (it >= budget) return 4;
    return 0;
}

// the WHILE condition of the captured loop: continue while no exit reason holds (at most ctl[1]
// iterations per graph launch, so the loop always ends)
__global__ void k_mr_check(const double* mr, double* ctl, cudaGraphConditionalHandle h) {
    pdl_wait();
    const double it = ctl[2] + 1.0;
    ctl[2] = it;
    const int r = mr_exit_reason(mr, ctl[0], it, ctl[1]);
    ctl[3] = double(r);
    cudaGraphSetConditional(h, r == 0 ? 1u : 0u);
}

// one MINRES iteration on fixed buffers V = {V0, V1, Zc, Zn, D1, D2, AZ}, iterate X
static void mr_iteration(pbm_grid* g, bool fp32, bool pc32, bool op_s, void* const* V, void* X, int64_t nv,
                         cudaStream_t st) {
    level_apply(g, 0, fp32, op_s, args(V[2], V[6], EPI_APPLY, nullptr, nullptr, nullptr, 0), st);
    mr_lanczos2(g, fp32, V[6], V[0], V[1], nv, st);
    precondition(g, fp32, pc32, op_s, V[1], V[3], nv, st);
    mr_scalars(g, st);
    mr_update2(g, fp32, V[2], V[3], V[4], V[5], X, nv, st);
}

// the captured loop for (fp32, op_s, pc32); built on first use
static cudaGraphExec_t mr_graph(pbm_grid* g, bool fp32, bool pc32, bool op_s, void* const* V, void* X, int64_t nv,
                                int64_t& kernels) {
    const int key = (fp32 ? 1 : 0) | (op_s ? 2 : 0) | (pc32 ? 4 : 0);
    kernels = g->mr_graph_kernels[key];
    if (g->mr_graph[key]) return g->mr_graph[key];
    if (!g->cap_stream) PBM_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t cs = g->cap_stream;
    cudaGraph_t graph = nullptr;
    PBM_CUDA(cudaGraphCreate(&graph, 0));
    const int64_t before = launch_count();
    try {
        cudaGraphConditionalHandle h;
        PBM_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        PBM_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        PBM_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        try {
            mr_iteration(g, fp32, pc32, op_s, V, X, nv, cs);
            launch_pdl(k_mr_check, dim3(1), dim3(1), 0, cs, g->sc->mr, g->sc->ctl, h);
            PBM_LAUNCH("mr check");
        } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(cs, &dummy);
            throw;
        }
        PBM_CUDA(cudaStreamEndCapture(cs, &body));
        cudaGraphExec_t ex = nullptr;
        PBM_CUDA(cudaGraphInstantiate(&ex, graph, 0));
        g->mr_graph[key] = ex;
    } catch (...) {
        cudaGraphDestroy(graph);
        count_launch_add(before - launch_count());
        throw;
    }
    cudaGraphDestroy(graph);
    // captured launches did not run: count them when the graph executes
    kernels = launch_count() - before;
    g->mr_graph_kernels[key] = kernels;
    count_launch_add(-kernels);
    return g->mr_graph[key];
}

static MrResult minres(pbm_grid* g, bool fp32, bool op_s, const void* b, void* x, double rtol, int maxit,
                       bool check_true, cudaStream_t st, bool pc32 = false) {
    MrResult res;
    const int64_t nv = g->L[0].g.n() + (op_s ? 1 : 0);
    void* const* V = fp32 ? (void* const*)g->kv32 : (void* const*)g->kv64;
    void* X = V[10];
    const size_t bytes = nv * esz(fp32);
    // |b|^2 and |x|^2 of the initial guess in one read; from x = 0 the starting residual is b itself (bit for bit)
    // and the operator application is skipped
    launch_dot(g, fp32, b, b, nv, 3, st);
    launch_dot(g, fp32, x, x, nv, 57, st);
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[3], &g->sc->red[3], sizeof(double), cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[57], &g->sc->red[57], sizeof(double), cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    const double bnorm = std::sqrt(g->sc_host->red[3]);
    const bool x_zero = g->sc_host->red[57] == 0.0;
    if (bnorm == 0.0) {
        vec_zero(x, bytes, st);
        return res;
    }
    auto finish = [&]() { PBM_CUDA(cudaMemcpyAsync(x, X, bytes, cudaMemcpyDeviceToDevice, st)); };
    if (x_zero) {
        // (a guess whose squares all underflow counts as zero: the iterate starts from exactly zero)
        vec_zero(X, bytes, st);
        PBM_CUDA(cudaMemcpyAsync(V[1], b, bytes, cudaMemcpyDeviceToDevice, st));
    } else {
        PBM_CUDA(cudaMemcpyAsync(X, x, bytes, cudaMemcpyDeviceToDevice, st));
        level_apply(g, 0, fp32, op_s, args(X, V[1], EPI_RESID, b, nullptr, nullptr, 2), st);
    }
    precondition(g, fp32, pc32, op_s, V[1], V[2], nv, st);
    mr_init(g, st);
    vec_zero(V[0], bytes, st);
    vec_zero(V[4], bytes, st);
    vec_zero(V[5], bytes, st);
    double target = rtol;
    double last_check = std::numeric_limits<double>::infinity();
    double* mr = g->sc_host->mr;
    double* ctl = g->sc_host->ctl;
    auto read_state = [&](bool with_ctl) {
        PBM_CUDA(cudaMemcpyAsync(mr, g->sc->mr, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
        if (with_ctl) PBM_CUDA(cudaMemcpyAsync(ctl, g->sc->ctl, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
    };
    read_state(false);
    if (mr[13] != 0.0) {
        res.status = PBM_EBREAKDOWN;
        finish();
        return res;
    }
    // the graph cannot hold the profiling event pairs: profiled solves launch eagerly
    const bool graph = !g->prof_on;
    while (res.iters < maxit) {
        int reason = 0;
        const int budget = maxit - res.iters;
        if (graph) {
            int64_t kernels = 0;
            cudaGraphExec_t ex = mr_graph(g, fp32, pc32, op_s, V, X, nv, kernels);
            launch_pdl(k_mr_ctl, dim3(1), dim3(1), 0, st, g->sc->ctl, target, double(budget));
            PBM_LAUNCH("mr ctl");
            PBM_CUDA(cudaGraphLaunch(ex, st));
            read_state(true);
            res.iters += int(ctl[2]);
            count_launch_add(kernels * int64_t(ctl[2]));
            reason = int(ctl[3]);
        } else {
            mr_iteration(g, fp32, pc32, op_s, V, X, nv, st);
            read_state(false);
            res.iters += 1;
            reason = mr[13] == 1.0 ? 1 : (mr[13] == 2.0 || mr[1] == 0.0) ? 2
                   : (std::fabs(mr[6]) <= target * mr[7]) ? 3 : (res.iters >= maxit ? 4 : 0);
        }
        if (reason == 1) {
            res.status = PBM_EBREAKDOWN;
            finish();
            return res;
        }
        if (reason == 2 || reason == 3) {
            if (!check_true) {
                finish();
                return res;
            }
            level_apply(g, 0, fp32, op_s, args(X, V[6], EPI_RESID, b, nullptr, nullptr, 2), st);
            res.relres = std::sqrt(read_slot(g, 2, st)) / bnorm;
            if (res.relres <= rtol) {
                finish();
                return res;
            }
            if (reason == 2 || !(res.relres < 0.5 * last_check)) {
                res.status = PBM_ENOTCONV;
                finish();
                return res;
            }
            last_check = res.relres;
            target = target * 0.5 * rtol / res.relres;
        }
    }
    if (check_true) {
        level_apply(g, 0, fp32, op_s, args(X, V[6], EPI_RESID, b, nullptr, nullptr, 2), st);
        res.relres = std::sqrt(read_slot(g, 2, st)) / bnorm;
        res.status = res.relres <= rtol ? PBM_OK : PBM_ENOTCONV;
    } else {
        res.status = PBM_ENOTCONV;
    }
    finish();
    return res;
}

// FP64 true residual relres of x for b (op on the fine level)
static double true_relres(pbm_grid* g, bool op_s, const double* b, const double* x, double* r, double bnorm,
                          cudaStream_t st) {
    level_apply(g, 0, false, op_s, args(x, r, EPI_RESID, b, nullptr, nullptr, 2), st);
    return std::sqrt(read_slot(g, 2, st)) / bnorm;
}

// Mixed precision (PBM_MIXED), two stages:
//  1. FP64 iterative refinement around inner MINRES solves of the residual equation that run
//     entirely in FP32 (operator, V-cycle, vectors; FP64 scalars) to desc.inner_rtol. Each step must
//     at least halve the FP64 residual; a step that does not is undone and the solve moves on.
//  2. FP64 MINRES (FP64 vectors and operator) preconditioned by the FP32 V-cycle, restarted from
//     the current iterate (residual replacement) while the true residual keeps halving. It needs
//     only the preconditioner to be accurate to FP32, so it also converges where the FP32
//     operator is too inexact for stage 1 (condition number near 1 / FP32 epsilon).
int solve(pbm_grid* g, bool op_s, const double* b, double* x, double rtol, int maxit, pbm_solve_info* info,
          cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    const int64_t nv = g->L[0].g.n() + (op_s ? 1 : 0);
    pbm_solve_info inf{};
    if (g->desc.precision == PBM_FP64) {
        MrResult r = minres(g, false, op_s, b, x, rtol, maxit, true, st);
        inf.status = r.status;
        inf.iterations = r.iters;
        inf.outer = 1;
        inf.relres = r.relres;
    } else {
        double* r64 = g->kv64[7];
        float* r32 = g->kv32[7];
        float* dx32 = g->kv32[8];
        // |b|^2 and |x|^2 of the initial guess in one read: from x = 0 the first FP64 residual is b itself (bit for
        // bit: the operator of zero is zero, supported rows give b - 0), so the FP64 apply is skipped
        launch_dot(g, false, b, b, nv, 3, st);
        launch_dot(g, false, x, x, nv, 57, st);
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[3], &g->sc->red[3], sizeof(double), cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[57], &g->sc->red[57], sizeof(double), cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
        const double bnorm = std::sqrt(g->sc_host->red[3]);
        const bool x_zero = g->sc_host->red[57] == 0.0;
        inf.status = PBM_OK;
        if (bnorm == 0.0) {
            vec_zero(x, nv * sizeof(double), st);
        } else {
            int total = 0, outer = 0;
            double rel;
            if (x_zero) {
                PBM_CUDA(cudaMemcpyAsync(r64, b, nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
                rel = 1.0;
            } else {
                rel = true_relres(g, op_s, b, x, r64, bnorm, st);
            }
            bool robust = false;
            while (rel > rtol && !robust) {
                if (total >= maxit || outer >= 60) break;
                ++outer;
                launch_cast(r64, false, r32, true, nv, st);
                vec_zero(dx32, nv * sizeof(float), st);
                MrResult ir = minres(g, true, op_s, r32, dx32, g->desc.inner_rtol, maxit - total, false, st);
                total += ir.iters;
                if (ir.status == PBM_EBREAKDOWN) {
                    robust = true;
                    break;
                }
                add_f32(x, dx32, nv, st, 1.0);
                const double prev = rel;
                rel = true_relres(g, op_s, b, x, r64, bnorm, st);
                if (!(rel < 0.5 * prev)) {
                    if (!(rel < prev)) {
                        add_f32(x, dx32, nv, st, -1.0);
                        rel = prev;
                    }
                    robust = true;
                }
            }
            double last = std::numeric_limits<double>::infinity();
            while (rel > rtol && robust && total < maxit) {
                ++outer;
                MrResult r = minres(g, false, op_s, b, x, rtol, maxit - total, true, st, true);
                total += r.iters;
                rel = r.relres;
                if (r.status == PBM_EBREAKDOWN) {
                    inf.status = PBM_EBREAKDOWN;
                    break;
                }
                if (r.status == PBM_OK || !(rel < 0.5 * last)) break;
                last = rel;
            }
            if (inf.status == PBM_OK && rel > rtol) inf.status = PBM_ENOTCONV;
            inf.iterations = total;
            inf.outer = outer;
            inf.relres = rel;
        }
    }
    inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return inf.status;
}

}  // namespace pbm
