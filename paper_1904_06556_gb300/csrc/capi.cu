// C ABI entry points (include/pbm.h): argument checks, allocation, and the sequencing of the
// kernels for each call.
#include <chrono>
#include <cmath>
#include <cstring>
#include <atomic>
#include <limits>

#include "pbm_internal.h"

namespace pbm {

void setup_hierarchy(pbm_grid* g, bool op_s, cudaStream_t st);
void vcycle(pbm_grid* g, int k, bool fp32, bool op_s, const void* b, void* x, int dot_slot, cudaStream_t st,
            bool first_done = false);
int solve(pbm_grid* g, bool op_s, const double* b, double* x, double rtol, int maxit, pbm_solve_info* info,
          cudaStream_t st);
void launch_coeffs(pbm_grid* g, const pbm_state* s, const double* c2, double* coef, cudaStream_t st);
void set_entry(double* y, int64_t i, const double* src, double a, double b, cudaStream_t st);
void launch_check_nonneg(pbm_grid* g, const double* v, int64_t n, int slot, cudaStream_t st);
void launch_mask_copy(pbm_grid* g, const double* x, double* y, cudaStream_t st);
void launch_delta_nu(pbm_grid* g, const double* bq, const double* coef, const double* dz_alpha, double* dl, double* du,
                     cudaStream_t st);
void launch_lagr_terms(pbm_grid* g, double kappa, const double* c2u, const double* bq, const double* qq,
                       const pbm_state* s, const double* dl, const double* dup, double alpha_k, int slot,
                       cudaStream_t st);
void launch_axpy(double* y, const double* x, double kappa, int64_t n, cudaStream_t st);
void launch_scale(const double* a, double* b, double s, int64_t n, cudaStream_t st);
void launch_mult_update(pbm_grid* g, const double* c2, pbm_state* s, double beta, bool only_rho, cudaStream_t st);
void launch_gap_sums(pbm_grid* g, const double* c2, const pbm_state* s, int slot, cudaStream_t st);
void launch_ip_coeffs(pbm_grid* g, const pbm_ip_state* s, const double* c2, double* coef, cudaStream_t st);
void launch_doc(pbm_grid* g, const double* e, double* rho_inout, double V, double rho_lo, double rho_up, double q,
                double tau, double* w, cudaStream_t st);
void launch_ip_recover(pbm_grid* g, const double* wdu, const double* da, const double* coef, double rho_lo,
                       double rho_up, double* drho, double* dnl, double* dnu, cudaStream_t st);

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launch_add(int64_t delta) { g_launches.fetch_add((long long)delta, std::memory_order_relaxed); }
int64_t launch_count() { return int64_t(g_launches.load(std::memory_order_relaxed)); }

int num_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];   // 0: not queried yet
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDev) fail(PBM_EINVAL, "device ordinal out of range");
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        check_cuda(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev), "SM count");
        if (v <= 0) fail(PBM_ECUDA, "device reports no SMs");
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// ------------------------------------------------------------------------------------------------
// profiling of the fine-level operator kernel: an event pair per launch, folded on read
// ------------------------------------------------------------------------------------------------
void prof_fold(pbm_grid* g) {
    if (g->prof_used == 0) return;
    PBM_CUDA(cudaEventSynchronize(g->prof_ev[2 * g->prof_used - 1]));
    for (size_t i = 0; i < g->prof_used; ++i) {
        float ms = 0.0f;
        PBM_CUDA(cudaEventElapsedTime(&ms, g->prof_ev[2 * i], g->prof_ev[2 * i + 1]));
        g->prof[g->prof_op[i]].total_ms += double(ms);
    }
    g->prof_used = 0;
}

void prof_begin(pbm_grid* g, cudaStream_t st) {
    if (!g->prof_on) return;
    if (g->prof_used * 2 == g->prof_ev.size()) {
        if (g->prof_ev.size() >= 2 * 4096) {
            prof_fold(g);  // pool full: wait for the recorded launches and reuse the events
        } else {
            for (int i = 0; i < 2 * 256; ++i) {
                cudaEvent_t e;
                PBM_CUDA(cudaEventCreate(&e));
                g->prof_ev.push_back(e);
            }
            g->prof_op.resize(g->prof_ev.size() / 2);
        }
    }
    PBM_CUDA(cudaEventRecord(g->prof_ev[2 * g->prof_used], st));
}

void prof_end(pbm_grid* g, cudaStream_t st, int op, double bytes, double flops) {
    if (!g->prof_on) return;
    PBM_CUDA(cudaEventRecord(g->prof_ev[2 * g->prof_used + 1], st));
    g->prof_op[g->prof_used] = op;
    ++g->prof_used;
    g->prof[op].launches += 1;
    g->prof[op].bytes += bytes;
    g->prof[op].flops += flops;
}

void set_error(const std::string& msg) { g_last_error = msg; }
void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(PBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dalloc(pbm_grid* g, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        fail(PBM_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    g->bytes += int64_t(bytes);
    return p;
}
void dfree(void* p) {
    if (p) cudaFree(p);
}

// ------------------------------------------------------------------------------------------------
// element matrix from the weak form: K^{cd}_{ab} = h [ lam M^{cd}_{ab} + mu M^{dc}_{ab}
//   + mu delta_cd sum_k M^{kk}_{ab} ],  M^{cd}_{ab} = int_{[0,1]^3} d_c N_a d_d N_b, a product over the
// three directions of 1D integrals: int N'N' = [[1,-1],[-1,1]], int NN = [[1/3,1/6],[1/6,1/3]],
// int N_a' N_b = [[-1/2,-1/2],[1/2,1/2]] (and its transpose for int N_a N_b').
// ------------------------------------------------------------------------------------------------
static void element_matrix(double E, double nu, double h, double* K) {
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    const double S1[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
    const double M1[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
    const double C1[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};
    auto Mcd = [&](int c, int d, int a, int b) {
        double v = 1.0;
        for (int k = 0; k < 3; ++k) {
            const int ia = (a >> k) & 1, ib = (b >> k) & 1;
            if (k == c && k == d) v *= S1[ia][ib];
            else if (k == c) v *= C1[ia][ib];
            else if (k == d) v *= C1[ib][ia];
            else v *= M1[ia][ib];
        }
        return v;
    };
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) {
                    double v = lam * Mcd(c, d, a, b) + mu * Mcd(d, c, a, b);
                    if (c == d) v += mu * (Mcd(0, 0, a, b) + Mcd(1, 1, a, b) + Mcd(2, 2, a, b));
                    K[(3 * a + c) * 24 + 3 * b + d] = h * v;
                }
}

void element_hat(double E, double nu, double h, KeHat& K) {
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    auto mm = [](int bit) { return bit ? 1.0 / 12.0 : 0.25; };
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 8; ++q) {
            double v = 0.0;
            if ((q >> c) & 1) {
                int o[2], n = 0;
                for (int k = 0; k < 3; ++k)
                    if (k != c) o[n++] = k;
                v += (lam + mu) * mm((q >> o[0]) & 1) * mm((q >> o[1]) & 1);
            }
            for (int k = 0; k < 3; ++k) {
                if (!((q >> k) & 1)) continue;
                double pr = 1.0;
                for (int j = 0; j < 3; ++j)
                    if (j != k) pr *= mm((q >> j) & 1);
                v += mu * pr;
            }
            K.dg[c][q] = h * v;
        }
    for (int b = 0; b < 2; ++b) {
        K.lam4[b] = h * lam * 0.25 * mm(b);
        K.mu4[b] = h * mu * 0.25 * mm(b);
    }
}

static double pcw(int c, int a, int A) {
    double w = 1.0;
    for (int k = 0; k < 3; ++k) {
        const int Ak = (A >> k) & 1, s = ((c >> k) & 1) + ((a >> k) & 1);
        w *= (s == 1) ? 0.5 : ((s == 0) ? (Ak == 0 ? 1.0 : 0.0) : (Ak == 1 ? 1.0 : 0.0));
    }
    return w;
}

struct StreamGuard {
    cudaStream_t st;
};

static cudaStream_t S(void* s) { return (cudaStream_t)s; }

static void set_device(const pbm_grid* g) { PBM_CUDA(cudaSetDevice(g->device)); }

}  // namespace pbm

using namespace pbm;

#define PBM_TRY try {
#define PBM_CATCH                                                       \
    }                                                                   \
    catch (const Error& e) {                                            \
        set_error(e.msg);                                               \
        return e.code;                                                  \
    }                                                                   \
    catch (const std::exception& e) {                                   \
        set_error(std::string("host exception: ") + e.what());          \
        return PBM_ENOMEM;                                              \
    }                                                                   \
    set_error("");                                                      \
    return PBM_OK;

extern "C" {

const char* pbm_last_error(void) { return g_last_error.c_str(); }

int pbm_default_desc(pbm_grid_desc* d, int nx, int ny, int nz, int levels, int support) {
    if (!d) {
        set_error("null desc");
        return PBM_EINVAL;
    }
    std::memset(d, 0, sizeof(*d));
    d->nx = nx;
    d->ny = ny;
    d->nz = nz;
    d->levels = levels;
    d->support = support;
    d->precision = PBM_FP64;
    d->E = 1.0;
    d->nu = 0.3;
    d->h = 1.0;
    d->pre_sweeps = 2;
    d->post_sweeps = 2;
    d->jacobi_theta = 1.2;
    d->lanczos_steps = 10;
    d->inner_rtol = 1e-4;
    d->smoother = PBM_SMOOTHER_JACOBI;
    set_error("");
    return PBM_OK;
}

int pbm_create_grid(const pbm_grid_desc* d, pbm_grid** out) {
    pbm_grid* g = nullptr;
    PBM_TRY
    if (!d || !out) fail(PBM_EINVAL, "null argument");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) fail(PBM_EINVAL, "grid dimensions must be >= 1");
    if (d->levels < 1 || d->levels > 16) fail(PBM_EINVAL, "levels must be in 1..16");
    const int f = 1 << (d->levels - 1);
    if (d->nx % f || d->ny % f || d->nz % f) fail(PBM_EINVAL, "nx, ny, nz must be divisible by 2^(levels-1)");
    if (d->support < PBM_CANTILEVER || d->support > PBM_FREE) fail(PBM_EINVAL, "unknown support");
    if (d->precision != PBM_FP64 && d->precision != PBM_MIXED) fail(PBM_EINVAL, "unknown precision");
    if (!(d->E > 0.0) || !(d->nu > -1.0 && d->nu < 0.5) || !(d->h > 0.0)) fail(PBM_EINVAL, "bad material or h");
    if (d->pre_sweeps < 0 || d->post_sweeps < 0 || d->pre_sweeps + d->post_sweeps < 1 || d->pre_sweeps > 64 ||
        d->post_sweeps > 64)
        fail(PBM_EINVAL, "sweeps must be in 0..64, at least one in total");
    if (!(d->jacobi_theta > 0.0 && d->jacobi_theta < 2.0)) fail(PBM_EINVAL, "jacobi_theta must be in (0, 2)");
    if (d->smoother != PBM_SMOOTHER_JACOBI && d->smoother != PBM_SMOOTHER_CHEBYSHEV &&
        d->smoother != PBM_SMOOTHER_GAUSS_SEIDEL)
        fail(PBM_EINVAL, "unknown smoother");
    if (d->smoother == PBM_SMOOTHER_CHEBYSHEV && (d->pre_sweeps > kChebMaxStep + 1 || d->post_sweeps > kChebMaxStep + 1))
        fail(PBM_EINVAL, "Chebyshev smoothing takes at most 9 steps per pass");
    if (d->lanczos_steps < 2 || d->lanczos_steps > 64) fail(PBM_EINVAL, "lanczos_steps must be in 2..64");
    if (d->precision == PBM_MIXED && !(d->inner_rtol > 0.0 && d->inner_rtol < 1.0))
        fail(PBM_EINVAL, "inner_rtol must be in (0, 1)");
    const int64_t nc_dofs = 3LL * (d->nx / f + 1) * (d->ny / f + 1) * (d->nz / f + 1);
    if (d->levels >= 2 && nc_dofs > 1500) fail(PBM_EINVAL, "coarsest grid too large (more than 1500 dofs): add levels");
    if (d->levels < 2) fail(PBM_EINVAL, "at least 2 levels are needed (the V-cycle ends in an exact coarse solve)");
    if (3.0 * (d->nx + 1.0) * (d->ny + 1.0) * (d->nz + 1.0) >= 2147483647.0 ||
        8.0 * double(d->nx) * d->ny * d->nz >= 2147483647.0)
        fail(PBM_EINVAL, "grid too large: the kernels index nodes and elements with 32-bit integers");

    g = new pbm_grid();
    g->desc = *d;
    PBM_CUDA(cudaGetDevice(&g->device));
    g->levels = d->levels;
    g->L.resize(d->levels);
    const bool mixed = d->precision == PBM_MIXED;
    for (int k = 0; k < d->levels; ++k) {
        Level& L = g->L[k];
        L.g = Geom{d->nx >> k, d->ny >> k, d->nz >> k, d->support};
        L.h = d->h * double(1 << k);
    }
    element_matrix(d->E, d->nu, d->h, g->Ke);
    element_hat(d->E, d->nu, d->h, g->kehat);
    g->Kdiag = g->Ke[0];
    // G_c = P_c^T K_e P_c
    std::vector<double> Gtri(8 * NTRI);
    for (int c = 0; c < 8; ++c) {
        for (int I = 0; I < 24; ++I)
            for (int J = 0; J < 24; ++J) {
                const int A = I / 3, ci = I % 3, B = J / 3, cj = J % 3;
                double s = 0.0;
                for (int a = 0; a < 8; ++a) {
                    const double wa = pcw(c, a, A);
                    if (wa == 0.0) continue;
                    for (int b = 0; b < 8; ++b) {
                        const double wb = pcw(c, b, B);
                        if (wb == 0.0) continue;
                        s += wa * wb * g->Ke[(3 * a + ci) * 24 + 3 * b + cj];
                    }
                }
                g->G[c][I * 24 + J] = s;
            }
        for (int i = 0; i < 24; ++i)
            for (int j = i; j < 24; ++j) Gtri[c * NTRI + tri_index(i, j)] = g->G[c][i * 24 + j];
    }
    g->G_dev = (double*)dalloc(g, sizeof(double) * 8 * NTRI);
    PBM_CUDA(cudaMemcpy(g->G_dev, Gtri.data(), sizeof(double) * 8 * NTRI, cudaMemcpyHostToDevice));
    if (g->desc.precision == PBM_MIXED) {
        std::vector<float> G32(Gtri.begin(), Gtri.end());
        g->G32 = (float*)dalloc(g, sizeof(float) * 8 * NTRI);
        PBM_CUDA(cudaMemcpy(g->G32, G32.data(), sizeof(float) * 8 * NTRI, cudaMemcpyHostToDevice));
    }
    {
        std::vector<float> B;
        tc_build(g->Ke, B, g->tc.terms, g->tc.scale);
        g->tcB = (float*)dalloc(g, sizeof(float) * B.size());
        PBM_CUDA(cudaMemcpy(g->tcB, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice));
        g->tc.B = g->tcB;
    }

    const Geom& F = g->L[0].g;
    const int64_t n = F.n(), m = F.m();
    for (int k = 0; k < d->levels; ++k) {
        Level& L = g->L[k];
        const int64_t nk = L.g.n() + 1, mk = L.g.m();
        if (k >= 1) {
            L.A64 = (double*)dalloc(g, sizeof(double) * NTRI * mk);
            if (mixed) L.A32 = (float*)dalloc(g, sizeof(float) * NTRI * mk);
            const size_t nq = size_t(12) * size_t(L.g.nx) * size_t(L.g.ny) * size_t(L.g.nz + 1);
            L.qa = dalloc(g, sizeof(double) * nq);
            L.qb = dalloc(g, sizeof(double) * nq);
        }
        L.bord64 = (double*)dalloc(g, sizeof(double) * nk);
        L.diag64 = (double*)dalloc(g, sizeof(double) * nk);
        L.idiag64 = (double*)dalloc(g, sizeof(double) * nk);
        L.sdiag64 = (double*)dalloc(g, sizeof(double) * nk);
        L.x64 = (double*)dalloc(g, sizeof(double) * nk);
        L.b64 = (double*)dalloc(g, sizeof(double) * nk);
        L.r64 = (double*)dalloc(g, sizeof(double) * nk);
        L.t64 = (double*)dalloc(g, sizeof(double) * nk);
        if (mixed) {
            L.bord32 = (float*)dalloc(g, sizeof(float) * nk);
            L.idiag32 = (float*)dalloc(g, sizeof(float) * nk);
            L.x32 = (float*)dalloc(g, sizeof(float) * nk);
            L.b32 = (float*)dalloc(g, sizeof(float) * nk);
            L.r32 = (float*)dalloc(g, sizeof(float) * nk);
            L.t32 = (float*)dalloc(g, sizeof(float) * nk);
        }
        PBM_CUDA(cudaMemset(L.bord64, 0, sizeof(double) * nk));
    }
    g->rho = (double*)dalloc(g, sizeof(double) * m);
    g->w64 = (double*)dalloc(g, sizeof(double) * m);
    g->d64 = (double*)dalloc(g, sizeof(double) * m);
    g->eps64 = (double*)dalloc(g, sizeof(double) * m);
    g->aux64 = (double*)dalloc(g, sizeof(double) * 8 * m);  // 5 coefficient rows + 3 line-search forms
    g->wr64 = (double*)dalloc(g, sizeof(double) * m);
    g->u64 = (double*)dalloc(g, sizeof(double) * (n + 1));
    g->what = (double*)dalloc(g, sizeof(double) * 24 * m);
    g->what_hat = (double*)dalloc(g, sizeof(double) * 21 * m);
    {
        const int64_t ncol = int64_t(d->nx) * d->ny;
        g->qa = dalloc(g, sizeof(double) * 12 * ncol * (d->nz + 1));
        g->qb = dalloc(g, sizeof(double) * 12 * ncol * d->nz);
    }
    g->nwt = (double*)dalloc(g, sizeof(double) * (2 * n + 1 + 2 * m));
    PBM_CUDA(cudaMemset(g->u64, 0, sizeof(double) * (n + 1)));
    if (mixed) {
        g->rho32 = (float*)dalloc(g, sizeof(float) * m);
        g->w32 = (float*)dalloc(g, sizeof(float) * m);
        g->d32 = (float*)dalloc(g, sizeof(float) * m);
        g->u32 = (float*)dalloc(g, sizeof(float) * (n + 1));
    }
    for (int i = 0; i < 12; ++i) {
        g->kv64[i] = (double*)dalloc(g, sizeof(double) * (n + 1));
        if (mixed) g->kv32[i] = (float*)dalloc(g, sizeof(float) * (n + 1));
    }
    g->nc = int(g->L[d->levels - 1].g.n());
    const size_t N = size_t(g->nc) + 1;
    g->cinv = (double*)dalloc(g, sizeof(double) * N * N);
    g->cwork = (double*)dalloc(g, sizeof(double) * (2 * N * N + N));   // L, L^{-1}, 1 / diag(L)
    g->max_blocks = 1 << 16;
    g->partials = (double*)dalloc(g, sizeof(double) * size_t(8 + 2 * (kRedSets - 1)) * size_t(g->max_blocks));
    g->sc = (DevScalars*)dalloc(g, sizeof(DevScalars));
    PBM_CUDA(cudaMemset(g->sc, 0, sizeof(DevScalars)));
    PBM_CUDA(cudaMallocHost((void**)&g->sc_host, sizeof(DevScalars)));
    std::memset(g->sc_host, 0, sizeof(DevScalars));
    PBM_CUDA(cudaDeviceSynchronize());
    g->fusedP[0] = g->fusedP[1] = fused_default_plan(g->L[0].g);
    autotune_fine(g);
    PBM_CUDA(cudaDeviceSynchronize());
    *out = g;
    g = nullptr;
    }
    catch (const Error& e) {
        set_error(e.msg);
        if (g) pbm_destroy_grid(g);
        return e.code;
    }
    set_error("");
    return PBM_OK;
}

int pbm_destroy_grid(pbm_grid* g) {
    if (!g) return PBM_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    for (auto& L : g->L) {
        dfree(L.A64);
        dfree(L.A32);
        dfree(L.qa);
        dfree(L.qb);
        dfree(L.bord64);
        dfree(L.bord32);
        dfree(L.diag64);
        dfree(L.idiag64);
        dfree(L.sdiag64);
        dfree(L.idiag32);
        dfree(L.x64);
        dfree(L.b64);
        dfree(L.r64);
        dfree(L.t64);
        dfree(L.x32);
        dfree(L.b32);
        dfree(L.r32);
        dfree(L.t32);
    }
    dfree(g->G_dev);
    dfree(g->G32);
    dfree(g->tcB);
    dfree(g->rho);
    dfree(g->w64);
    dfree(g->d64);
    dfree(g->eps64);
    dfree(g->aux64);
    dfree(g->wr64);
    dfree(g->rho32);
    dfree(g->w32);
    dfree(g->d32);
    dfree(g->u64);
    dfree(g->u32);
    dfree(g->what);
    dfree(g->what_hat);
    dfree(g->qa);
    dfree(g->qb);
    dfree(g->nwt);
    for (int i = 0; i < 12; ++i) {
        dfree(g->kv64[i]);
        dfree(g->kv32[i]);
    }
    for (cudaGraphExec_t e : g->mr_graph)
        if (e) cudaGraphExecDestroy(e);
    dfree(g->ip_work);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (auto& sst : g->side)
        if (sst) cudaStreamDestroy(sst);
    for (auto& ev : g->side_ev)
        if (ev) cudaEventDestroy(ev);
    dfree(g->cinv);
    dfree(g->cwork);
    dfree(g->partials);
    dfree(g->sc);
    for (cudaEvent_t e : g->prof_ev) cudaEventDestroy(e);
    if (g->sc_host) cudaFreeHost(g->sc_host);
    delete g;
    return PBM_OK;
}

int pbm_grid_info_get(const pbm_grid* g, pbm_grid_info* out) {
    PBM_TRY
    if (!g || !out) fail(PBM_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->levels = g->levels;
    for (int k = 0; k < g->levels; ++k) {
        out->nx[k] = g->L[k].g.nx;
        out->ny[k] = g->L[k].g.ny;
        out->nz[k] = g->L[k].g.nz;
        out->n[k] = g->L[k].g.n();
        out->m[k] = g->L[k].g.m();
        out->omega[k] = g->L[k].omega;
        out->lambda_max[k] = g->L[k].lambda_max;
    }
    const Geom& F = g->L[0].g;
    // supported nodes: every support lies on the faces x = 0 and x = nx, so only those are visited
    int64_t fixed = 0;
    for (int k = 0; k <= F.nz; ++k)
        for (int j = 0; j <= F.ny; ++j) {
            fixed += node_fixed(F.support, F.nx, F.ny, F.nz, 0, j, k) ? 1 : 0;
            if (F.nx > 0) fixed += node_fixed(F.support, F.nx, F.ny, F.nz, F.nx, j, k) ? 1 : 0;
        }
    out->n_free = F.n() - 3 * fixed;
    out->device_bytes = g->bytes;
    out->fine_chunk[0] = fine_L(g, false, false);
    out->fine_chunk[1] = fine_L(g, false, true);
    out->fine_chunk[2] = g->desc.precision == PBM_MIXED ? fine_L(g, true, false) : 0;
    out->fine_chunk[3] = g->desc.precision == PBM_MIXED ? fine_L(g, true, true) : 0;
    for (int op = 0; op < 2; ++op) {
        const FusedPlan fp = fused_plan(F, g->fusedP[op], op == 1);
        out->fp32_tile[op][0] = fp.TX;
        out->fp32_tile[op][1] = fp.TY;
        out->fp32_tile[op][2] = fp.DZ;
        out->fp32_tile[op][3] = fused_threads(fp);
        out->fp32_tile[op][4] = g->fusedP[op];
        if (g->desc.precision == PBM_MIXED)
            for (int k = 1; k + 1 < g->levels; ++k) out->coarse_plan[op][k] = g->coarseP[op][k];
    }
    PBM_CATCH
}

int pbm_get_maps(const pbm_grid* g, int level, int which, void* host_dst) {
    PBM_TRY
    if (!g || !host_dst) fail(PBM_EINVAL, "null argument");
    if (level < 0 || level >= g->levels) fail(PBM_EINVAL, "bad level");
    const Geom& G = g->L[level].g;
    const int sx = G.nx + 1, sxy = (G.nx + 1) * (G.ny + 1);
    if (which == PBM_MAP_FIXED_DOFS) {
        uint8_t* o = (uint8_t*)host_dst;
        for (int k = 0; k <= G.nz; ++k)
            for (int j = 0; j <= G.ny; ++j)
                for (int i = 0; i <= G.nx; ++i) {
                    const int64_t nd = i + int64_t(sx) * j + int64_t(sxy) * k;
                    const uint8_t fx = node_fixed(G.support, G.nx, G.ny, G.nz, i, j, k) ? 1 : 0;
                    o[3 * nd] = o[3 * nd + 1] = o[3 * nd + 2] = fx;
                }
    } else if (which == PBM_MAP_ELEM_NODES) {
        int32_t* o = (int32_t*)host_dst;
        for (int64_t e = 0; e < G.m(); ++e) {
            const int i = int(e % G.nx), j = int((e / G.nx) % G.ny), k = int(e / (int64_t(G.nx) * G.ny));
            for (int a = 0; a < 8; ++a)
                o[8 * e + a] = int32_t((i + (a & 1)) + int64_t(sx) * (j + ((a >> 1) & 1)) + int64_t(sxy) * (k + (a >> 2)));
        }
    } else if (which == PBM_MAP_PROLONG) {
        if (level < 1) fail(PBM_EINVAL, "PBM_MAP_PROLONG needs level >= 1");
        const Geom& Fg = g->L[level - 1].g;
        const int64_t nnf = Fg.nnode();
        int32_t* ids = (int32_t*)host_dst;
        double* wts = (double*)(ids + 8 * nnf);
        const int csx = G.nx + 1, csxy = (G.nx + 1) * (G.ny + 1);
        for (int64_t fn = 0; fn < nnf; ++fn) {
            const int I = int(fn % (Fg.nx + 1)), J = int((fn / (Fg.nx + 1)) % (Fg.ny + 1)),
                      K = int(fn / (int64_t(Fg.nx + 1) * (Fg.ny + 1)));
            int slot = 0;
            for (int kc = K >> 1; kc <= (K + 1) >> 1; ++kc)
                for (int jc = J >> 1; jc <= (J + 1) >> 1; ++jc)
                    for (int ic = I >> 1; ic <= (I + 1) >> 1; ++ic) {
                        const double w = ((I & 1) ? 0.5 : 1.0) * ((J & 1) ? 0.5 : 1.0) * ((K & 1) ? 0.5 : 1.0);
                        ids[8 * fn + slot] = int32_t(ic + int64_t(csx) * jc + int64_t(csxy) * kc);
                        wts[8 * fn + slot] = w;
                        ++slot;
                    }
            for (; slot < 8; ++slot) {
                ids[8 * fn + slot] = -1;
                wts[8 * fn + slot] = 0.0;
            }
        }
    } else if (which == PBM_MAP_KE) {
        const double s = double(1 << level);
        double* o = (double*)host_dst;
        for (int i = 0; i < 576; ++i) o[i] = s * g->Ke[i];
    } else {
        fail(PBM_EINVAL, "unknown map");
    }
    PBM_CATCH
}

int pbm_set_density(pbm_grid* g, const double* rho_dev, void* stream) {
    PBM_TRY
    if (!g || !rho_dev) fail(PBM_EINVAL, "null argument");
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t m = g->L[0].g.m();
    PBM_CUDA(cudaMemcpyAsync(g->rho, rho_dev, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    launch_check_nonneg(g, g->rho, m, 13, st);
    const double bad = read_slot(g, 13, st);
    if (bad != 0.0) fail(PBM_ENONFINITE, "density has non-finite or negative entries");
    g->rho_set = true;
    if (g->op_ready == 1) g->op_ready = 0;
    PBM_CATCH
}

int pbm_apply_K(pbm_grid* g, const double* w_dev, const double* x_dev, double* y_dev, int level, void* stream) {
    PBM_TRY
    if (!g || !x_dev || !y_dev) fail(PBM_EINVAL, "null argument");
    if (level < 0 || level >= g->levels) fail(PBM_EINVAL, "level out of range");
    if (level > 0 && w_dev) fail(PBM_EINVAL, "coarse levels apply the Galerkin operators of the set density: w must be NULL");
    if (!w_dev && !g->rho_set) fail(PBM_ESTATE, "no density set");
    set_device(g);
    const cudaStream_t st = S(stream);
    ApplyArgs a{};
    a.x = x_dev;
    a.y = y_dev;
    a.mode = EPI_APPLY;
    a.dot_slot = -1;
    if (level == 0) {
        launch_fine(g, false, w_dev ? w_dev : g->rho, nullptr, nullptr, a, st);
    } else {
        // the Galerkin chain of K(rho) (Section 5.1): built here if no K solve or V-cycle has built it
        if (g->op_ready != 1) setup_hierarchy(g, false, st);
        ensure_coarse64(g, st);
        launch_coarse(g, level, false, a, st);
    }
    PBM_CATCH
}

int pbm_apply_K_f32(pbm_grid* g, const float* w_dev, const float* x_dev, float* y_dev, void* stream) {
    PBM_TRY
    if (!g || !x_dev || !y_dev || !w_dev) fail(PBM_EINVAL, "null argument");
    set_device(g);
    ApplyArgs a{};
    a.x = x_dev;
    a.y = y_dev;
    a.mode = EPI_APPLY;
    a.dot_slot = -1;
    launch_fine(g, true, w_dev, nullptr, nullptr, a, S(stream));
    PBM_CATCH
}

int pbm_apply_fine_f32(pbm_grid* g, int op, int epilogue, const float* x_dev, const float* b_dev, float* y_dev,
                       double* dot_host, void* stream) {
    return pbm_apply_level_f32(g, 0, op, epilogue, x_dev, b_dev, y_dev, dot_host, stream);
}

int pbm_apply_level_f32(pbm_grid* g, int level, int op, int epilogue, const float* x_dev, const float* b_dev,
                        float* y_dev, double* dot_host, void* stream) {
    PBM_TRY
    if (!g || !x_dev || !y_dev) fail(PBM_EINVAL, "null argument");
    if (level < 0 || level >= g->levels) fail(PBM_EINVAL, "level out of range");
    if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
    if (epilogue < PBM_EPI_APPLY || epilogue > PBM_EPI_JACOBI) fail(PBM_EINVAL, "unknown epilogue");
    if (epilogue != PBM_EPI_APPLY && !b_dev) fail(PBM_EINVAL, "the residual and Jacobi epilogues need b");
    if (g->desc.precision != PBM_MIXED) fail(PBM_ESTATE, "FP32 operators need a PBM_MIXED grid");
    if (g->op_ready != (op == PBM_OP_S ? 2 : 1)) fail(PBM_ESTATE, "the operator's hierarchy is not set up");
    set_device(g);
    const cudaStream_t st = S(stream);
    ApplyArgs a{};
    a.x = x_dev;
    a.y = y_dev;
    a.b = b_dev;
    a.diag = g->L[level].idiag32;
    a.omega = &g->sc->mr[16 + level];
    a.mode = epilogue;
    a.dot_slot = dot_host ? 56 : -1;
    level_apply(g, level, true, op == PBM_OP_S, a, st);
    if (dot_host) *dot_host = read_slot(g, 56, st);
    PBM_CATCH
}

int pbm_fp32_plan_count(void) { return fused_num_plans(); }

int pbm_fp32_tc_plan(void) { return fused_tc_plan(); }

int pbm_set_fp32_plan(pbm_grid* g, int op, int plan) {
    PBM_TRY
    if (!g) fail(PBM_EINVAL, "null grid");
    if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
    if (plan < 0 || plan >= fused_num_plans()) fail(PBM_EINVAL, "plan out of range");
    g->fusedP[op == PBM_OP_S ? 1 : 0] = plan;
    PBM_CATCH
}

int pbm_fp32_coarse_plan_count(void) { return fused_coarse_num_plans(); }

int pbm_set_fp32_coarse_plan(pbm_grid* g, int op, int level, int plan) {
    PBM_TRY
    if (!g) fail(PBM_EINVAL, "null grid");
    if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
    if (g->desc.precision != PBM_MIXED) fail(PBM_ESTATE, "FP32 operators need a PBM_MIXED grid");
    if (level < 1 || level > g->levels - 2) fail(PBM_EINVAL, "not a coarse level with an operator");
    if (plan < -2 || plan >= fused_coarse_num_plans()) fail(PBM_EINVAL, "plan out of range");
    g->coarseP[op == PBM_OP_S ? 1 : 0][level] = plan;
    PBM_CATCH
}

int pbm_get_diag(const pbm_grid* g, int level, double* diag_dev, void* stream) {
    PBM_TRY
    if (!g || !diag_dev) fail(PBM_EINVAL, "null argument");
    if (level < 0 || level >= g->levels) fail(PBM_EINVAL, "level out of range");
    if (g->op_ready == 0) fail(PBM_ESTATE, "no hierarchy has been set up");
    set_device(const_cast<pbm_grid*>(g));
    const Level& L = g->L[level];
    if (level >= 1) ensure_coarse64(const_cast<pbm_grid*>(g), S(stream));
    PBM_CUDA(cudaMemcpyAsync(diag_dev, L.diag64, sizeof(double) * (L.g.n() + 1), cudaMemcpyDeviceToDevice,
                             S(stream)));
    PBM_CATCH
}

static void check_state(const pbm_state* st) {
    if (!st || !st->u_dev || !st->nu_lo_dev || !st->nu_up_dev || !st->rho_dev || !st->mu_lo_dev || !st->mu_up_dev)
        fail(PBM_EINVAL, "null state array");
    if (!(st->p > 0.0) || !(st->q_lo > 0.0) || !(st->q_up > 0.0)) fail(PBM_EINVAL, "penalties must be > 0");
}

int pbm_set_state(pbm_grid* g, const pbm_state* s, void* stream) {
    PBM_TRY
    if (!g) fail(PBM_EINVAL, "null grid");
    check_state(s);
    set_device(g);
    const cudaStream_t st = S(stream);
    // coefficient rows live after the (rho' - eps) row: aux64 = [coef(5m) | c2 | b | q]
    const int64_t m = g->L[0].g.m();
    launch_mask_copy(g, s->u_dev, g->u64, st);
    double* c2 = g->aux64 + 5 * m;
    launch_elem_energy(g, g->u64, nullptr, c2, st);
    launch_coeffs(g, s, c2, g->aux64, st);
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[8], &g->sc->red[8], sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    if (g->sc_host->red[12] != 0.0) fail(PBM_ENONFINITE, "non-finite or non-positive Newton coefficients");
    g->s_alpha = g->sc_host->red[8];
    PBM_CUDA(cudaMemcpyAsync(&g->sc->salpha, &g->sc->red[8], sizeof(double), cudaMemcpyDeviceToDevice, st));
    g->sum_rho1 = g->sc_host->red[9];
    g->sum_wr = g->sc_host->red[10];
    g->gl2 = g->sc_host->red[11];
    g->alpha = s->alpha;
    g->V = s->V;
    g->state_set = true;
    g->ip_set = false;
    setup_hierarchy(g, true, st);
    PBM_CATCH
}

// ------------------------------------------------------------------------------------------------
// interior-point Newton system (Section 4.1). S_IP = Jf S Jf with Jf = diag(I, -1) and S the PBM-form
// operator (border -1) built from w = rho and the weights d: the applies and the solve flip the
// sign of the alpha entry around the PBM-form kernels.
// ------------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------------
// damped optimality criteria (Algorithm DOC)
// ------------------------------------------------------------------------------------------------
int pbm_default_doc_params(pbm_doc_params* p) {
    if (!p) return PBM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->rho_up = 1.0;
    p->q = 0.5;
    p->eps_doc = 1e-3;
    p->tau_alpha = 0.0;
    p->eps_mr = 1e-4;
    p->maxit = 500;
    p->max_iter = 1000;
    return PBM_OK;
}

static void doc_iteration(pbm_grid* g, double* rho_dev, const double* f_dev, double* u_dev, const pbm_doc_params* p,
                          pbm_doc_info* info, cudaStream_t st) {
    const int64_t m = g->L[0].g.m(), n = g->L[0].g.n();
    // rho into the handle (checked), then the equilibrium solve on the K(rho) hierarchy
    PBM_CUDA(cudaMemcpyAsync(g->rho, rho_dev, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    launch_check_nonneg(g, g->rho, m, 13, st);
    if (read_slot(g, 13, st) != 0.0) fail(PBM_ENONFINITE, "density has non-finite or negative entries");
    g->rho_set = true;
    setup_hierarchy(g, false, st);
    pbm_solve_info inf{};
    const int rc = solve(g, false, f_dev, u_dev, p->eps_mr, p->maxit, &inf, st);
    info->minres += inf.iterations;
    info->minres_relres = inf.relres;
    if (rc != PBM_OK) fail(rc, rc == PBM_EBREAKDOWN ? "MINRES breakdown" : "equilibrium solve did not converge");
    double* e = g->aux64 + 6 * m;
    double* w = g->aux64 + 7 * m;
    launch_elem_energy(g, u_dev, nullptr, e, st);
    const double tau = p->tau_alpha > 0.0 ? p->tau_alpha : 0.1 * p->eps_doc;
    launch_doc(g, e, rho_dev, p->V, p->rho_lo, p->rho_up, p->q, tau, w, st);
    launch_dot(g, false, f_dev, u_dev, n, 14, st);
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[12], &g->sc->red[12], sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->ctl[0], &g->sc->ctl[0], sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    info->change = g->sc_host->red[12];
    info->compliance = g->sc_host->red[14];
    info->alpha = g->sc_host->ctl[2];
    info->trials = int(g->sc_host->ctl[3]);
    info->iterations += 1;
}

static void check_doc(pbm_grid* g, const double* rho_dev, const double* f_dev, const double* u_dev,
                      const pbm_doc_params* p) {
    if (!g || !rho_dev || !f_dev || !u_dev || !p) fail(PBM_EINVAL, "null argument");
    if (!(p->rho_up > p->rho_lo) || !(p->rho_lo >= 0.0)) fail(PBM_EINVAL, "need 0 <= rho_lo < rho_up");
    if (!(p->q > 0.0) || !(p->eps_mr > 0.0) || p->maxit < 1) fail(PBM_EINVAL, "need q > 0, eps_mr > 0, maxit >= 1");
    if (!(p->tau_alpha > 0.0) && !(p->eps_doc > 0.0)) fail(PBM_EINVAL, "need tau_alpha > 0 or eps_doc > 0");
    if (!(p->V > 0.0)) fail(PBM_EINVAL, "need V > 0");
}

int pbm_doc_step(pbm_grid* g, double* rho_dev, const double* f_dev, double* u_dev, const pbm_doc_params* p,
                 pbm_doc_info* info, void* stream) {
    PBM_TRY
    check_doc(g, rho_dev, f_dev, u_dev, p);
    set_device(g);
    pbm_doc_info inf{};
    doc_iteration(g, rho_dev, f_dev, u_dev, p, &inf, S(stream));
    if (info) *info = inf;
    PBM_CATCH
}

int pbm_doc_solve(pbm_grid* g, double* rho_dev, const double* f_dev, double* u_dev, const pbm_doc_params* p,
                  pbm_doc_info* info, void* stream) {
    pbm_doc_info inf{};
    int rc = PBM_OK;
    try {
        check_doc(g, rho_dev, f_dev, u_dev, p);
        if (!(p->eps_doc > 0.0) || p->max_iter < 1) fail(PBM_EINVAL, "need eps_doc > 0 and max_iter >= 1");
        set_device(g);
        const cudaStream_t st = S(stream);
        const int64_t m = g->L[0].g.m();
        double* prev = (double*)dalloc(g, sizeof(double) * m);
        try {
            bool done = false;
            while (!done && inf.iterations < p->max_iter) {
                // keep rho: Algorithm DOC stops with the density whose update was below the tolerance
                PBM_CUDA(cudaMemcpyAsync(prev, rho_dev, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
                doc_iteration(g, rho_dev, f_dev, u_dev, p, &inf, st);
                if (inf.change <= p->eps_doc) {
                    PBM_CUDA(cudaMemcpyAsync(rho_dev, prev, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
                    PBM_CUDA(cudaStreamSynchronize(st));
                    done = true;
                }
            }
            if (!done) fail(PBM_ENOTCONV, "DOC did not reach eps_doc in max_iter iterations");
        } catch (...) {
            cudaStreamSynchronize(st);
            dfree(prev);
            g->bytes -= int64_t(sizeof(double) * m);
            throw;
        }
        dfree(prev);
        g->bytes -= int64_t(sizeof(double) * m);
    } catch (const Error& e) {
        set_error(e.msg);
        rc = e.code;
    }
    inf.status = rc;
    if (info) *info = inf;
    if (rc == PBM_OK) set_error("");
    return rc;
}

static double* ip_work(pbm_grid* g) {
    if (!g->ip_work) g->ip_work = (double*)dalloc(g, sizeof(double) * 2 * size_t(g->L[0].g.n() + 1));
    return g->ip_work;
}

int pbm_ip_set_state(pbm_grid* g, const pbm_ip_state* s, void* stream) {
    PBM_TRY
    if (!g || !s || !s->u_dev || !s->rho_dev || !s->nu_lo_dev || !s->nu_up_dev) fail(PBM_EINVAL, "null argument");
    if (!(s->r > 0.0) || !(s->s > 0.0)) fail(PBM_EINVAL, "barrier parameters must be > 0");
    if (!(s->rho_up > s->rho_lo)) fail(PBM_EINVAL, "rho_up must exceed rho_lo");
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t m = g->L[0].g.m();
    ip_work(g);
    launch_mask_copy(g, s->u_dev, g->u64, st);
    double* c2 = g->aux64 + 5 * m;
    launch_elem_energy(g, g->u64, nullptr, c2, st);
    launch_ip_coeffs(g, s, c2, g->aux64, st);
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[8], &g->sc->red[8], sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    if (g->sc_host->red[10] != 0.0) fail(PBM_EINVAL, "interior-point state not strictly feasible or not finite");
    g->s_alpha = g->sc_host->red[8];
    PBM_CUDA(cudaMemcpyAsync(&g->sc->salpha, &g->sc->red[8], sizeof(double), cudaMemcpyDeviceToDevice, st));
    g->alpha = s->alpha;
    g->V = s->V;
    g->ip_rho_lo = s->rho_lo;
    g->ip_rho_up = s->rho_up;
    g->state_set = false;
    g->ip_set = true;
    setup_hierarchy(g, true, st);
    PBM_CATCH
}

static void require_ip(const pbm_grid* g) {
    if (!g->ip_set) fail(PBM_ESTATE, "pbm_ip_set_state has not been called");
}

int pbm_ip_apply_S(pbm_grid* g, const double* x_dev, double* y_dev, void* stream) {
    PBM_TRY
    if (!g || !x_dev || !y_dev) fail(PBM_EINVAL, "null argument");
    require_ip(g);
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n();
    double* xf = ip_work(g);
    PBM_CUDA(cudaMemcpyAsync(xf, x_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    set_entry(xf, n, x_dev + n, -1.0, 0.0, st);
    ApplyArgs a{};
    a.x = xf;
    a.y = y_dev;
    a.mode = EPI_APPLY;
    a.with_alpha = true;
    a.dot_slot = -1;
    launch_fine(g, false, g->w64, g->d64, g->u64, a, st);
    set_entry(y_dev, n, y_dev + n, -1.0, 0.0, st);
    PBM_CATCH
}

int pbm_ip_reduced_rhs(pbm_grid* g, const double* f_dev, double* rhs_dev, void* stream) {
    PBM_TRY
    if (!g || !f_dev || !rhs_dev) fail(PBM_EINVAL, "null argument");
    require_ip(g);
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n();
    // rhs_u = f - K(rho + d c) u (supported rows: f - u = 0); rhs_alpha = V - sum(rho + d c)
    ApplyArgs a{};
    a.x = g->u64;
    a.y = rhs_dev;
    a.b = f_dev;
    a.mode = EPI_RESID;
    a.dot_slot = -1;
    launch_fine(g, false, g->wr64, nullptr, nullptr, a, st);
    set_entry(rhs_dev, n, &g->sc->red[9], -1.0, g->V, st);
    PBM_CATCH
}

int pbm_ip_solve(pbm_grid* g, const double* rhs_dev, double* dz_dev, double rtol, int maxit, pbm_solve_info* info,
                 void* stream) {
    PBM_TRY
    if (!g || !rhs_dev || !dz_dev) fail(PBM_EINVAL, "null argument");
    if (!(rtol > 0.0) || maxit < 1) fail(PBM_EINVAL, "rtol must be > 0 and maxit >= 1");
    require_ip(g);
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n();
    auto t0 = std::chrono::steady_clock::now();
    if (g->op_ready != 2) setup_hierarchy(g, true, st);
    const double setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    // the PBM-form system S (Jf dz) = Jf rhs
    double* bf = ip_work(g) + (n + 1);
    PBM_CUDA(cudaMemcpyAsync(bf, rhs_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    set_entry(bf, n, rhs_dev + n, -1.0, 0.0, st);
    set_entry(dz_dev, n, dz_dev + n, -1.0, 0.0, st);
    pbm_solve_info inf{};
    const int rc = solve(g, true, bf, dz_dev, rtol, maxit, &inf, st);
    set_entry(dz_dev, n, dz_dev + n, -1.0, 0.0, st);
    inf.setup_ms = setup_ms;
    if (info) *info = inf;
    if (rc != PBM_OK) {
        set_error(rc == PBM_EBREAKDOWN ? "MINRES breakdown: preconditioner not positive definite"
                                       : "MINRES did not reach the tolerance");
        return rc;
    }
    PBM_CATCH
}

int pbm_ip_recover(pbm_grid* g, const double* dz_dev, double* drho_dev, double* dnu_lo_dev, double* dnu_up_dev,
                   void* stream) {
    PBM_TRY
    if (!g || !dz_dev || !drho_dev || !dnu_lo_dev || !dnu_up_dev) fail(PBM_EINVAL, "null argument");
    require_ip(g);
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t m = g->L[0].g.m(), n = g->L[0].g.n();
    double* wdu = g->aux64 + 6 * m;
    launch_elem_energy(g, g->u64, dz_dev, wdu, st);
    launch_ip_recover(g, wdu, dz_dev + n, g->aux64, g->ip_rho_lo, g->ip_rho_up, drho_dev, dnu_lo_dev, dnu_up_dev, st);
    PBM_CATCH
}

int pbm_apply_S(pbm_grid* g, const double* x_dev, double* y_dev, void* stream) {
    PBM_TRY
    if (!g || !x_dev || !y_dev) fail(PBM_EINVAL, "null argument");
    if (!g->state_set) fail(PBM_ESTATE, "pbm_set_state has not been called");
    set_device(g);
    ApplyArgs a{};
    a.x = x_dev;
    a.y = y_dev;
    a.mode = EPI_APPLY;
    a.with_alpha = true;
    a.dot_slot = -1;
    launch_fine(g, false, g->w64, g->d64, g->u64, a, S(stream));
    PBM_CATCH
}

int pbm_reduced_rhs(pbm_grid* g, const double* f_dev, double* rhs_dev, double* norms_host, void* stream) {
    PBM_TRY
    if (!g || !f_dev || !rhs_dev) fail(PBM_EINVAL, "null argument");
    if (!g->state_set) fail(PBM_ESTATE, "pbm_set_state has not been called");
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n();
    // rhs_u = f - K(rho' - eps) u (supported rows: f - u = 0); rhs_alpha = -V + sum (rho' - eps)
    ApplyArgs a{};
    a.x = g->u64;
    a.y = rhs_dev;
    a.b = f_dev;
    a.mode = EPI_RESID;
    a.dot_slot = -1;
    launch_fine(g, false, g->wr64, nullptr, nullptr, a, st);
    set_entry(rhs_dev, n, &g->sc->red[10], 1.0, -g->V, st);
    if (norms_host) {
        // res_1 = K(rho') u - f on free dofs: ||f - K(rho') u||
        ApplyArgs b{};
        b.x = g->u64;
        b.y = g->kv64[8];
        b.b = f_dev;
        b.mode = EPI_RESID;
        b.dot_slot = 4;
        launch_fine(g, false, g->w64, nullptr, nullptr, b, st);
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[0], &g->sc->red[0], sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
        norms_host[0] = std::sqrt(g->sc_host->red[4]);
        norms_host[1] = g->V - g->sum_rho1;
        norms_host[2] = std::sqrt(g->gl2);
    }
    PBM_CATCH
}

int pbm_vcycle(pbm_grid* g, int op, const double* b_dev, double* x_dev, void* stream) {
    PBM_TRY
    if (!g || !b_dev || !x_dev) fail(PBM_EINVAL, "null argument");
    if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
    set_device(g);
    const cudaStream_t st = S(stream);
    const bool op_s = op == PBM_OP_S;
    if (op_s) {
        if (!g->state_set) fail(PBM_ESTATE, "pbm_set_state has not been called");
        if (g->op_ready != 2) {
            // the K hierarchy replaced it: rebuild S's (coefficients are still in place)
            setup_hierarchy(g, true, st);
        }
    } else {
        if (!g->rho_set) fail(PBM_ESTATE, "no density set");
        if (g->op_ready != 1) setup_hierarchy(g, false, st);
    }
    const int64_t nv = g->L[0].g.n() + (op_s ? 1 : 0);
    if (g->desc.precision == PBM_MIXED) {
        float* b32 = g->kv32[7];
        float* x32 = g->kv32[8];
        launch_cast(b_dev, false, b32, true, nv, st);
        vcycle(g, 0, true, op_s, b32, x32, -1, st);
        launch_cast(x32, true, x_dev, false, nv, st);
    } else {
        vcycle(g, 0, false, op_s, b_dev, x_dev, -1, st);
    }
    PBM_CATCH
}

int pbm_minres_solve(pbm_grid* g, int op, const double* b_dev, double* x_dev, double rtol, int maxit,
                     pbm_solve_info* info, void* stream) {
    PBM_TRY
    if (!g || !b_dev || !x_dev) fail(PBM_EINVAL, "null argument");
    if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
    if (!(rtol > 0.0) || maxit < 1) fail(PBM_EINVAL, "rtol must be > 0 and maxit >= 1");
    set_device(g);
    const cudaStream_t st = S(stream);
    const bool op_s = op == PBM_OP_S;
    auto t0 = std::chrono::steady_clock::now();
    double setup_ms = 0.0;
    if (op_s) {
        if (!g->state_set) fail(PBM_ESTATE, "pbm_set_state has not been called");
        if (g->op_ready != 2) setup_hierarchy(g, true, st);
    } else {
        if (!g->rho_set) fail(PBM_ESTATE, "no density set");
        if (g->op_ready != 1) setup_hierarchy(g, false, st);
    }
    setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    pbm_solve_info inf{};
    const int rc = solve(g, op_s, b_dev, x_dev, rtol, maxit, &inf, st);
    inf.setup_ms = setup_ms;
    if (info) *info = inf;
    if (rc != PBM_OK) {
        set_error(rc == PBM_EBREAKDOWN ? "MINRES breakdown: preconditioner not positive definite"
                                       : "MINRES did not reach the tolerance");
        return rc;
    }
    PBM_CATCH
}

// One Newton step of Algorithm 2 (see pbm_newton_step). With eps_stop > 0 the step is not taken
// when res_PBM at the current state is already below eps_stop (*stepped = false). Returns the MINRES
// status of the step (PBM_OK or PBM_ENOTCONV); throws on every other error.
// With res_prev >= 0 the MINRES tolerance adapts before the solve (Section 5.3): if res_PBM has not
// fallen below 0.9 res_prev, *eps_mr = max(*eps_mr / 10, eps_mr_min).
// A direction with grad L^T dxi >= 0 (not one of descent; Section 6 reports such directions from
// inexact solves near the end of its largest runs) is solved again from zero with eps_mr / 10, down
// to eps_mr_min; the tightened tolerance is kept (*eps_mr). If the direction is still not one of
// descent at the floor the step is not taken: inf.stalled = 1, *stepped = false, PBM_ELINESEARCH.
static int newton_core(pbm_grid* g, pbm_state* s, const double* f_dev, double* eps_mr_io, double eps_stop,
                       pbm_newton_info& inf, void* stream, bool* stepped, double res_prev, double eps_mr_min,
                       int max_halvings, int maxit) {
    int rc_solve = PBM_OK;
    *stepped = false;
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n(), m = g->L[0].g.m();
    int rc = pbm_set_state(g, s, stream);
    if (rc != PBM_OK) fail(rc, pbm_last_error());
    double* dz = g->nwt;
    double* r = dz + n + 1;
    double* dl = r + n;
    double* dup = dl + m;
    double* rhs = g->kv64[9];
    double norms[3];
    rc = pbm_reduced_rhs(g, f_dev, rhs, norms, stream);
    if (rc != PBM_OK) fail(rc, pbm_last_error());
    launch_dot(g, false, f_dev, f_dev, n, 20, st);
    const double fnorm = std::sqrt(read_slot(g, 20, st));
    const double rho_n = std::sqrt(double(m)) * (std::fabs(s->rho_lo) + std::fabs(s->rho_up));
    inf.res_pbm = norms[0] / fnorm + std::fabs(norms[1]) / s->V + norms[2] / rho_n;
    if (eps_stop > 0.0 && inf.res_pbm < eps_stop) return PBM_OK;
    if (res_prev >= 0.0 && inf.res_pbm > 0.9 * res_prev) *eps_mr_io = std::max(0.1 * *eps_mr_io, eps_mr_min);
    double eps_mr = *eps_mr_io;
    double* c2 = g->aux64 + 5 * m;
    double* bq = g->aux64 + 6 * m;
    double* qq = g->aux64 + 7 * m;
    // grad_u L = K(rho') u - f = -(f - K(rho') u), a function of the state only
    {
        ApplyArgs a{};
        a.x = g->u64;
        a.y = r;
        a.b = f_dev;
        a.mode = EPI_RESID;
        a.dot_slot = -1;
        launch_fine(g, false, g->w64, nullptr, nullptr, a, st);
    }
    launch_dot(g, false, f_dev, g->u64, n, 28, st);
    const double g_alpha = s->V - g->sum_rho1;
    double slope = 0.0, dalpha = 0.0, fTu = 0.0, fTdu = 0.0;
    for (;;) {
        // reduced Newton system S dz = rhs (eq. (system)), from zero
        PBM_CUDA(cudaMemsetAsync(dz, 0, sizeof(double) * (n + 1), st));
        pbm_solve_info si{};
        rc_solve = solve(g, true, rhs, dz, eps_mr, maxit, &si, st);
        inf.minres_iterations += si.iterations;
        inf.minres_relres = si.relres;
        if (rc_solve == PBM_EBREAKDOWN) fail(PBM_EBREAKDOWN, "MINRES breakdown in the Newton system");
        // per-element forms b = u^T K_e du, q = du^T K_e du; nu-step (eq. (deltanu))
        launch_elem_energy(g, g->u64, dz, bq, st);
        launch_elem_energy(g, dz, nullptr, qq, st);
        launch_delta_nu(g, bq, g->aux64, dz + n, dl, dup, st);
        // directional derivative grad L . dxi
        launch_dot(g, false, r, dz, n, 21, st);
        launch_dot(g, false, g->aux64 + 3 * m, dl, m, 22, st);
        launch_dot(g, false, g->aux64 + 4 * m, dup, m, 23, st);
        launch_dot(g, false, f_dev, dz, n, 29, st);
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[20], &g->sc->red[20], sizeof(double) * 12, cudaMemcpyDeviceToHost,
                                 st));
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->ctl[7], dz + n, sizeof(double), cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
        const double* R = g->sc_host->red;
        dalpha = g->sc_host->ctl[7];
        slope = -R[21] + g_alpha * dalpha + R[22] + R[23];
        fTu = R[28];
        fTdu = R[29];
        if (slope < 0.0 || eps_mr <= eps_mr_min) break;
        eps_mr = std::max(0.1 * eps_mr, eps_mr_min);
        inf.resolves += 1;
    }
    *eps_mr_io = eps_mr;
    inf.eps_mr = eps_mr;
    inf.slope = slope;
    if (!(slope < 0.0)) {
        inf.stalled = 1;
        fail(PBM_ELINESEARCH, "no descent direction at the MINRES tolerance floor: the Newton step is not taken");
    }
    auto lagr = [&](double kappa) {
        launch_lagr_terms(g, kappa, c2, bq, qq, s, dl, dup, s->alpha + kappa * dalpha, 24, st);
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[24], &g->sc->red[24], sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
        const double* T = g->sc_host->red + 24;
        if (T[3] != 0.0) return std::numeric_limits<double>::infinity();
        return (s->alpha + kappa * dalpha) * s->V - fTu - kappa * fTdu - s->rho_lo * T[1] + s->rho_up * T[2] + T[0];
    };
    const double L0 = lagr(0.0);
    inf.lagrangian_old = L0;
    double kappa = 1.0;
    bool ok = false;
    for (int h = 0; h <= max_halvings; ++h) {
        const double Lk = lagr(kappa);
        if (std::isfinite(Lk) && Lk <= L0 + 1e-4 * kappa * slope) {
            inf.lagrangian_new = Lk;
            inf.halvings = h;
            ok = true;
            break;
        }
        kappa *= 0.5;
    }
    if (!ok) fail(PBM_ELINESEARCH, "Armijo backtracking found no acceptable step");
    inf.kappa = kappa;
    launch_axpy(s->u_dev, dz, kappa, n, st);
    launch_axpy(s->nu_lo_dev, dl, kappa, m, st);
    launch_axpy(s->nu_up_dev, dup, kappa, m, st);
    s->alpha += kappa * dalpha;
    PBM_CUDA(cudaStreamSynchronize(st));
    *stepped = true;
    return rc_solve;
}

int pbm_default_newton_params(pbm_newton_params* p) {
    if (!p) {
        set_error("null argument");
        return PBM_EINVAL;
    }
    p->eps_mr = 1e-4;
    p->eps_mr_min = 1e-9;
    p->max_halvings = 30;
    p->maxit = 10000;
    set_error("");
    return PBM_OK;
}

int pbm_newton_step_ex(pbm_grid* g, pbm_state* s, const double* f_dev, const pbm_newton_params* prm,
                       pbm_newton_info* info, void* stream) {
    pbm_newton_info inf{};
    int rc_solve = PBM_OK;
    PBM_TRY
    if (!g || !f_dev || !prm) fail(PBM_EINVAL, "null argument");
    check_state(s);
    if (!(prm->eps_mr > 0.0) || !(prm->eps_mr_min > 0.0) || prm->max_halvings < 0 || prm->maxit < 1)
        fail(PBM_EINVAL, "eps_mr and eps_mr_min must be > 0, max_halvings >= 0, maxit >= 1");
    set_device(g);
    bool stepped = false;
    double eps_mr_v = prm->eps_mr;
    rc_solve = newton_core(g, s, f_dev, &eps_mr_v, -1.0, inf, stream, &stepped, -1.0,
                           std::min(prm->eps_mr_min, prm->eps_mr), prm->max_halvings, prm->maxit);
    inf.status = rc_solve;
    if (info) *info = inf;
    if (rc_solve != PBM_OK) {
        set_error("Newton step taken with an inexact solve (MINRES did not reach eps_mr)");
        return rc_solve;
    }
    }
    catch (const Error& e) {
        set_error(e.msg);
        inf.status = e.code;
        if (info) *info = inf;
        return e.code;
    }
    set_error("");
    return PBM_OK;
}

int pbm_newton_step(pbm_grid* g, pbm_state* s, const double* f_dev, double eps_mr, pbm_newton_info* info,
                    void* stream) {
    pbm_newton_params prm;
    pbm_default_newton_params(&prm);
    prm.eps_mr = eps_mr;
    return pbm_newton_step_ex(g, s, f_dev, &prm, info, stream);
}

int pbm_default_pbm_params(pbm_pbm_params* p) {
    if (!p) {
        set_error("null argument");
        return PBM_EINVAL;
    }
    p->eps_pbm = 1e-5;
    p->beta = 0.3;
    p->gamma = 0.3;
    p->p_min = 1e-8;
    p->eps_nwt = 1.0;
    p->eps_nwt_min = 1e-3;
    p->eps_mr = 0.0;
    p->eps_mr_min = 1e-9;
    p->max_outer = 100;
    p->max_newton = 100;
    p->max_halvings = 30;
    set_error("");
    return PBM_OK;
}

int pbm_solve(pbm_grid* g, pbm_state* s, const double* f_dev, const pbm_pbm_params* prm, pbm_pbm_info* info,
              void* stream) {
    pbm_pbm_info inf{};
    PBM_TRY
    if (!g || !f_dev || !prm) fail(PBM_EINVAL, "null argument");
    check_state(s);
    if (!(prm->beta > 0.0 && prm->beta < 1.0) || !(prm->gamma > 0.0 && prm->gamma < 1.0) || !(prm->p_min > 0.0) ||
        !(prm->eps_pbm > 0.0) || !(prm->eps_nwt > 0.0) || !(prm->eps_nwt_min > 0.0) || prm->max_outer < 1 ||
        prm->max_newton < 1 || prm->max_halvings < 0 || !(prm->eps_mr_min > 0.0))
        fail(PBM_EINVAL, "invalid PBM parameters");
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n(), m = g->L[0].g.m();
    double eps_nwt = prm->eps_nwt;
    double eps_mr = prm->eps_mr > 0.0 ? prm->eps_mr : 1e-4 * std::sqrt(double(g->L[0].g.n()));
    eps_mr = std::min(eps_mr, 0.5);
    double* c2 = g->aux64 + 5 * m;
    // Newton loop of Algorithm 2 to res_PBM < eps, adapting eps_MR (Section 5.3): when a step does not
    // reduce res_PBM below 0.9 of the previous value, eps_MR = max(eps_MR / 10, eps_mr_min)
    auto newton_loop = [&](double eps) {
        double res_prev = -1.0;
        for (int it = 0; it < prm->max_newton; ++it) {
            pbm_newton_info ni{};
            bool stepped = false;
            try {
                // a solve that stopped at maxit still gave a descent direction (checked in newton_core)
                (void)newton_core(g, s, f_dev, &eps_mr, eps, ni, stream, &stepped, res_prev, prm->eps_mr_min,
                                  prm->max_halvings, 10000);
            } catch (const Error& e) {
                inf.resolves += ni.resolves;
                inf.minres += ni.minres_iterations;
                if (e.code == PBM_ELINESEARCH && ni.stalled) {
                    // no descent direction even at eps_mr_min: the loop ends at the current iterate, which
                    // Section 6 accepts as the nearly optimal solution of a stalled run
                    inf.stalls += 1;
                    return;
                }
                throw;
            }
            inf.resolves += ni.resolves;
            inf.minres += ni.minres_iterations;
            if (!stepped) return;
            inf.newton += 1;
            res_prev = ni.res_pbm;
        }
        fail(PBM_ENOTCONV, "Newton loop reached max_newton steps");
    };
    // duality gap (eq. gap) and dual objective at the current state
    auto gap_ratio = [&](double& gap, double& dual) {
        launch_mask_copy(g, s->u_dev, g->u64, st);
        launch_elem_energy(g, g->u64, nullptr, c2, st);
        launch_gap_sums(g, c2, s, 30, st);
        launch_dot(g, false, f_dev, g->u64, n, 34, st);
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[30], &g->sc->red[30], sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
        const double* R = g->sc_host->red;
        const double fTu = R[34];
        gap = -0.5 * fTu + s->alpha * s->V - R[30];
        dual = s->alpha * s->V - fTu - s->rho_lo * R[31] + s->rho_up * R[32];
        inf.compliance = 0.5 * fTu;
        inf.volume = R[33];
        return std::fabs(gap / dual);
    };
    double ratio = std::numeric_limits<double>::infinity();
    for (int outer = 1; outer <= prm->max_outer; ++outer) {
        inf.outer = outer;
        newton_loop(eps_nwt);
        double gap = 0.0, dual = 0.0;
        ratio = gap_ratio(gap, dual);
        inf.gap_ratio = ratio;
        if (ratio < prm->eps_pbm) break;
        launch_mult_update(g, c2, s, prm->beta, false, st);
        s->p = std::max(prm->gamma * s->p, prm->p_min);
        s->q_lo = std::max(prm->gamma * s->q_lo, prm->p_min);
        s->q_up = std::max(prm->gamma * s->q_up, prm->p_min);
        eps_nwt = std::max(std::min(100.0 * ratio, eps_nwt), prm->eps_nwt_min);
    }
    // final Newton loop at 10 eps_PBM and the final density update of Algorithm 1
    newton_loop(10.0 * prm->eps_pbm);
    launch_mask_copy(g, s->u_dev, g->u64, st);
    launch_elem_energy(g, g->u64, nullptr, c2, st);
    launch_mult_update(g, c2, s, prm->beta, true, st);
    double gap = 0.0, dual = 0.0;
    (void)gap_ratio(gap, dual);
    inf.eps_mr = eps_mr;
    inf.status = ratio < prm->eps_pbm ? PBM_OK : PBM_ENOTCONV;
    if (info) *info = inf;
    if (inf.status != PBM_OK) {
        set_error("PBM reached max_outer iterations");
        return inf.status;
    }
    }
    catch (const Error& e) {
        set_error(e.msg);
        inf.status = e.code;
        if (info) *info = inf;
        return e.code;
    }
    set_error("");
    return PBM_OK;
}

int64_t pbm_kernel_launches(void) { return int64_t(g_launches.load(std::memory_order_relaxed)); }

int pbm_profile(pbm_grid* g, int on) {
    PBM_TRY
    if (!g) fail(PBM_EINVAL, "null grid");
    set_device(g);
    g->prof_on = on != 0;
    PBM_CATCH
}

int pbm_profile_read(pbm_grid* g, int op, pbm_profile_stats* out) {
    PBM_TRY
    if (!g || !out) fail(PBM_EINVAL, "null argument");
    if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
    set_device(g);
    prof_fold(g);
    *out = g->prof[op];
    g->prof[op] = pbm_profile_stats{};
    PBM_CATCH
}

int pbm_compliance_grad(pbm_grid* g, const double* u_dev, double* c_dev, const double* f_dev, double* fTu_host,
                        void* stream) {
    PBM_TRY
    if (!g || !u_dev || !c_dev) fail(PBM_EINVAL, "null argument");
    set_device(g);
    const cudaStream_t st = S(stream);
    const int64_t n = g->L[0].g.n(), m = g->L[0].g.m();
    double* um = g->kv64[9];
    launch_mask_copy(g, u_dev, um, st);
    launch_elem_energy(g, um, nullptr, c_dev, st);
    launch_scale(c_dev, c_dev, 0.5, m, st);
    if (f_dev && fTu_host) {
        launch_dot(g, false, f_dev, um, n, 5, st);
        *fTu_host = read_slot(g, 5, st);
    }
    PBM_CATCH
}

}  // extern "C"
