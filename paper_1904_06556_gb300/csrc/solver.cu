// Host orchestration of the multigrid-preconditioned MINRES solve (Section 5): hierarchy set-up,
// the V-cycle, the Lanczos estimate of the Jacobi weights, MINRES, and the mixed-precision
// iterative refinement. Every step runs in the kernels of apply.cu, mg.cu and krylov.cu; the host
// only sequences launches and reads back scalars.
#include <chrono>
#include <cmath>

#include "pbm_internal.h"

namespace pbm {

void mr_lanczos(pbm_grid* g, bool fp32, const void* Az, const void* vcur, void* vprev_next, int64_t n, cudaStream_t st);
void mr_scalars(pbm_grid* g, cudaStream_t st);
void mr_init(pbm_grid* g, cudaStream_t st);
void mr_update(pbm_grid* g, bool fp32, const void* z, void* d2, const void* d1, void* x, int64_t n, cudaStream_t st);
void add_f32(double* x, const float* d, int64_t n, cudaStream_t st);
void lz_start(pbm_grid* g, double* v, double* t, double* vprev, const double* diag, int64_t n, cudaStream_t st);
void lz_a(pbm_grid* g, double* w, const double* v, const double* diag, int64_t n, int j, cudaStream_t st);
void lz_b(pbm_grid* g, double* w, const double* v, const double* vprev, int64_t n, int j, cudaStream_t st);
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

// ------------------------------------------------------------------------------------------------
// V-cycle: x = M^{-1} b on level k (x overwritten). If dot_slot >= 0, red[dot_slot] = x . b.
// ------------------------------------------------------------------------------------------------
void vcycle(pbm_grid* g, int k, bool fp32, bool op_s, const void* b, void* x, int dot_slot, cudaStream_t st) {
    Level& L = g->L[k];
    const int64_t nv = L.g.n() + (op_s ? 1 : 0);
    if (k == g->levels - 1) {
        launch_coarsest_solve(g, fp32, b, x, op_s, st);
        if (dot_slot >= 0) launch_dot(g, fp32, x, b, nv, dot_slot, st);
        return;
    }
    void* t = fp32 ? (void*)L.t32 : (void*)L.t64;
    void* r = fp32 ? (void*)L.r32 : (void*)L.r64;
    const void* D = fp32 ? (const void*)L.diag32 : (const void*)L.diag64;
    const double* om = &g->sc->mr[16 + k];
    const int pre = g->desc.pre_sweeps, post = g->desc.post_sweeps;
    // pre-smoothing from x = 0: the first sweep is x = omega D^-1 b; arrange the ping-pong so that
    // the last pre-sweep lands in x
    void* cur = (pre % 2 == 1) ? x : t;
    void* oth = (cur == x) ? t : x;
    if (pre >= 1) {
        launch_scale_diag_first(g, k, fp32, b, cur, op_s, st);
        for (int s = 1; s < pre; ++s) {
            level_apply(g, k, fp32, op_s, args(cur, oth, EPI_JACOBI, b, D, om), st);
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
    launch_restrict(g, k, fp32, r, bc, op_s, 1.0, st);
    vcycle(g, k + 1, fp32, op_s, bc, xc, -1, st);
    launch_prolong_add(g, k, fp32, xc, x, op_s, st);
    // post-smoothing
    cur = x;
    oth = t;
    for (int s = 0; s < post; ++s) {
        const bool last = (s == post - 1);
        level_apply(g, k, fp32, op_s, args(cur, oth, EPI_JACOBI, b, D, om, last ? dot_slot : -1), st);
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

static void lanczos_level(pbm_grid* g, int k, bool op_s, cudaStream_t st) {
    Level& L = g->L[k];
    const int64_t nv = L.g.n() + (op_s ? 1 : 0);
    double* v = g->kv64[6];
    double* vp = g->kv64[7];
    double* t = g->kv64[8];
    double* w = g->kv64[9];
    const int steps = g->desc.lanczos_steps;
    lz_start(g, v, t, vp, L.diag64, nv, st);
    for (int j = 0; j < steps; ++j) {
        level_apply(g, k, false, op_s, args(t, w, EPI_APPLY), st);
        lz_a(g, w, v, L.diag64, nv, j, st);
        lz_b(g, w, v, vp, nv, j, st);
        lz_next(g, w, v, vp, t, L.diag64, nv, j, st);
    }
    PBM_CUDA(cudaMemcpyAsync(g->sc_host->lz_a, g->sc->lz_a, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaMemcpyAsync(g->sc_host->lz_b, g->sc->lz_b, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    std::vector<double> a, b;
    for (int j = 0; j < steps; ++j) {
        a.push_back(g->sc_host->lz_a[j]);
        const double bj = g->sc_host->lz_b[j];
        if (!(bj > 0.0) || j == steps - 1) break;
        b.push_back(bj);
    }
    b.resize(a.size() > 0 ? a.size() - 1 : 0);
    L.lambda_max = tridiag_max_eig(a, b);
    if (!(L.lambda_max > 0.0) || !std::isfinite(L.lambda_max)) fail(PBM_ENONFINITE, "Lanczos estimate is not positive");
    L.omega = g->desc.jacobi_theta / L.lambda_max;
}

static void upload_omegas(pbm_grid* g, cudaStream_t st) {
    for (int k = 0; k < g->levels; ++k) g->sc_host->mr[16 + k] = g->L[k].omega;
    PBM_CUDA(cudaMemcpyAsync(&g->sc->mr[16], &g->sc_host->mr[16], sizeof(double) * 16, cudaMemcpyHostToDevice, st));
}

// ------------------------------------------------------------------------------------------------
// hierarchy set-up for K(w64) (op_s = false) or S (op_s = true; coefficients already in place)
// ------------------------------------------------------------------------------------------------
void setup_hierarchy(pbm_grid* g, bool op_s, cudaStream_t st) {
    const bool mixed = g->desc.precision == PBM_MIXED;
    const int nl = g->levels;
    Level& F = g->L[0];
    if (op_s) {
        // alpha border of the fine level: b_0 = -sum_i d_i K_i u (restricted below with scale -1)
        launch_fine(g, false, g->d64, nullptr, nullptr, args(g->u64, F.bord64, EPI_APPLY), st);
        launch_build_what(g, st);
    } else {
        // K(w): what is not needed (d = 0); keep u zero so that nothing stale is used
    }
    launch_diag(g, 0, op_s, st);
    if (nl >= 2) {
        launch_build_level1(g, op_s, st);
        if (op_s) launch_restrict(g, 0, false, F.bord64, g->L[1].bord64, false, -1.0, st);
        for (int k = 1; k + 1 < nl; ++k) {
            launch_build_coarser(g, k, st);
            if (op_s) launch_restrict(g, k, false, g->L[k].bord64, g->L[k + 1].bord64, false, 1.0, st);
        }
        for (int k = 1; k < nl; ++k) launch_diag(g, k, op_s, st);
        build_coarsest(g, op_s, st);
    }
    if (mixed) {
        if (op_s) {
            launch_cast(g->w64, false, g->w32, true, F.g.m(), st);
            launch_cast(g->d64, false, g->d32, true, F.g.m(), st);
            launch_cast(g->u64, false, g->u32, true, F.g.n(), st);
        }
        else {
            launch_cast(g->rho, false, g->rho32, true, F.g.m(), st);
        }
        for (int k = 1; k < nl; ++k) launch_coarse_to_f32(g, k, st);
    }
    for (int k = 0; k + 1 < nl; ++k) lanczos_level(g, k, op_s, st);
    upload_omegas(g, st);
    // coarsest factorisation status
    PBM_CUDA(cudaMemcpyAsync(g->sc_host->flags, g->sc->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    if (nl >= 2 && g->sc_host->flags[0] != 0) fail(PBM_ENONFINITE, "coarsest matrix is not positive definite");
    g->op_ready = op_s ? 2 : 1;
}

// ------------------------------------------------------------------------------------------------
// MINRES (x holds the initial guess); returns status
// ------------------------------------------------------------------------------------------------
struct MrResult {
    int status = PBM_OK;
    int iters = 0;
    double relres = 0.0;
};

static MrResult minres(pbm_grid* g, bool fp32, bool op_s, const void* b, void* x, double rtol, int maxit,
                       bool check_true, cudaStream_t st) {
    MrResult res;
    const int64_t nv = g->L[0].g.n() + (op_s ? 1 : 0);
    void* const* pool = fp32 ? (void* const*)g->kv32 : (void* const*)g->kv64;
    void *vp = pool[0], *vc = pool[1], *z = pool[2], *z2 = pool[3], *dp = pool[4], *dp2 = pool[5], *Az = pool[6];
    const size_t bytes = nv * esz(fp32);
    launch_dot(g, fp32, b, b, nv, 3, st);
    const double bnorm = std::sqrt(read_slot(g, 3, st));
    if (bnorm == 0.0) {
        vec_zero(x, bytes, st);
        return res;
    }
    level_apply(g, 0, fp32, op_s, args(x, vc, EPI_RESID, b, nullptr, nullptr, 2), st);
    vcycle(g, 0, fp32, op_s, vc, z, 1, st);
    mr_init(g, st);
    vec_zero(vp, bytes, st);
    vec_zero(dp, bytes, st);
    vec_zero(dp2, bytes, st);
    double target = rtol;
    auto read_mr = [&]() {
        PBM_CUDA(cudaMemcpyAsync(g->sc_host->mr, g->sc->mr, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
    };
    read_mr();
    if (g->sc_host->mr[13] != 0.0) {
        res.status = PBM_EBREAKDOWN;
        return res;
    }
    const double r0 = std::sqrt(g->sc_host->red[2]);
    (void)r0;
    for (int it = 1; it <= maxit; ++it) {
        level_apply(g, 0, fp32, op_s, args(z, Az, EPI_APPLY, nullptr, nullptr, nullptr, 0), st);
        mr_lanczos(g, fp32, Az, vc, vp, nv, st);
        vcycle(g, 0, fp32, op_s, vp, z2, 1, st);
        mr_scalars(g, st);
        mr_update(g, fp32, z, dp2, dp, x, nv, st);
        std::swap(vp, vc);
        std::swap(dp2, dp);
        std::swap(z, z2);
        res.iters = it;
        read_mr();
        const double* mr = g->sc_host->mr;
        if (mr[13] == 1.0) {
            res.status = PBM_EBREAKDOWN;
            break;
        }
        const bool lucky = (mr[13] == 2.0) || mr[1] == 0.0;
        if (std::fabs(mr[6]) <= target * mr[7] || lucky) {
            if (!check_true) return res;
            level_apply(g, 0, fp32, op_s, args(x, Az, EPI_RESID, b, nullptr, nullptr, 2), st);
            res.relres = std::sqrt(read_slot(g, 2, st)) / bnorm;
            if (res.relres <= rtol || lucky) {
                res.status = res.relres <= rtol ? PBM_OK : PBM_ENOTCONV;
                return res;
            }
            target = target * 0.5 * rtol / res.relres;
        }
    }
    if (res.status == PBM_OK) {
        if (check_true) {
            level_apply(g, 0, fp32, op_s, args(x, Az, EPI_RESID, b, nullptr, nullptr, 2), st);
            res.relres = std::sqrt(read_slot(g, 2, st)) / bnorm;
            res.status = res.relres <= rtol ? PBM_OK : PBM_ENOTCONV;
        } else {
            res.status = PBM_ENOTCONV;
        }
    }
    return res;
}

// FP64 true residual relres of x for b (op on the fine level)
static double true_relres(pbm_grid* g, bool op_s, const double* b, const double* x, double* r, double bnorm,
                          cudaStream_t st) {
    level_apply(g, 0, false, op_s, args(x, r, EPI_RESID, b, nullptr, nullptr, 2), st);
    return std::sqrt(read_slot(g, 2, st)) / bnorm;
}

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
        // FP64 iterative refinement around FP32 MG-MINRES solves of the residual equation
        double* r64 = g->kv64[0];
        float* r32 = g->kv32[7];
        float* dx32 = g->kv32[8];
        launch_dot(g, false, b, b, nv, 3, st);
        const double bnorm = std::sqrt(read_slot(g, 3, st));
        inf.status = PBM_OK;
        if (bnorm == 0.0) {
            vec_zero(x, nv * sizeof(double), st);
        } else {
            int total = 0;
            double rel = true_relres(g, op_s, b, x, r64, bnorm, st);
            int outer = 0;
            while (rel > rtol) {
                if (total >= maxit || outer >= 60) {
                    inf.status = PBM_ENOTCONV;
                    break;
                }
                ++outer;
                launch_cast(r64, false, r32, true, nv, st);
                vec_zero(dx32, nv * sizeof(float), st);
                MrResult ir = minres(g, true, op_s, r32, dx32, g->desc.inner_rtol, maxit - total, false, st);
                total += ir.iters;
                if (ir.status == PBM_EBREAKDOWN) {
                    inf.status = PBM_EBREAKDOWN;
                    break;
                }
                add_f32(x, dx32, nv, st);
                const double prev = rel;
                rel = true_relres(g, op_s, b, x, r64, bnorm, st);
                if (!(rel < prev)) {  // no progress: stop rather than loop
                    inf.status = PBM_ENOTCONV;
                    break;
                }
            }
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
