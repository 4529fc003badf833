// Batched MG-MINRES: several independent systems (grid handles of any sizes, each with its operator
// set up) advanced together, one launch per stage of the MINRES iteration and the V-cycle.
//
// Each stage is one kernel launch over the CTAs of all systems that take part in it: a prefix table
// maps a CTA to (system, local CTA) and every system keeps its own buffers, scratch and device
// scalars. Systems of different depth share the stages down to their own coarsest level (the
// stage list is generated by walking the V-cycle recursion for all systems at once: at each depth
// the systems whose coarsest level it is get the dense coarse solve, the others smooth, restrict and
// recurse). A system whose MINRES has finished is marked inactive and its CTAs return at once. One
// iteration plus a check stage (exit reason per system, loop condition = some system active) is
// captured as the body of a CUDA graph WHILE node, so the loop runs without the host.
#include <chrono>
#include <cmath>
#include <limits>

#include "pbm_internal.h"

namespace pbm {

void launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, cudaStream_t st);
void add_f32(double* x, const float* d, int64_t n, cudaStream_t st, double sign);
void launch_dot(pbm_grid* g, bool fp32, const void* a, const void* b, int64_t n, int slot, cudaStream_t st);
int solve(pbm_grid* g, bool op_s, const double* b, double* x, double rtol, int maxit, pbm_solve_info* info,
          cudaStream_t st);

__device__ __forceinline__ int mr_exit_reason_b(const double* mr, double target, double it, double budget) {
    if (mr[13] == 1.0) return 1;
    if (mr[13] == 2.0 || mr[1] == 0.0) return 2;
    if (fabs(mr[6]) <= target * mr[7]) return 3;
    if (it >= budget) return 4;
    return 0;
}

// loop control of the batched graph: per system one more iteration, its exit reason, and the WHILE
// condition = some system still active (the iteration budget bounds every system, so it ends)
__global__ void k_batch_check(DevScalars* const* __restrict__ sc, int nsys, cudaGraphConditionalHandle h) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
        DevScalars* S = sc[s];
        if (S->flags[1] == 0) continue;
        const double it = S->ctl[2] + 1.0;
        S->ctl[2] = it;
        const int r = mr_exit_reason_b(S->mr, S->ctl[0], it, S->ctl[1]);
        S->ctl[3] = double(r);
        if (r != 0) S->flags[1] = 0;
        else atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// per system: ctl[0] target, ctl[1] budget, ctl[2] = 0, ctl[3] = 0, flags[1] = active (from `in`)
__global__ void k_batch_ctl(DevScalars* const* __restrict__ sc, int nsys, const double* __restrict__ in) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    DevScalars* S = sc[s];
    S->ctl[0] = in[3 * s];
    S->ctl[1] = in[3 * s + 1];
    S->ctl[2] = 0.0;
    S->ctl[3] = 0.0;
    S->flags[1] = in[3 * s + 2] != 0.0 ? 1 : 0;
}

// per system: iterations, exit reason, eta, eta0, status, red[2] (residual^2), red[3] (b.b)
constexpr int GATHER = 8;
__global__ void k_batch_gather(DevScalars* const* __restrict__ sc, int nsys, double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const DevScalars* S = sc[s];
    double* o = out + GATHER * s;
    o[0] = S->ctl[2];
    o[1] = S->ctl[3];
    o[2] = S->mr[6];
    o[3] = S->mr[7];
    o[4] = S->mr[13];
    o[5] = S->red[2];
    o[6] = S->red[3];
    o[7] = S->mr[1];
}

enum StageKind { ST_FINE, ST_COARSE, ST_NODES, ST_RESTRICT, ST_PROLONG, ST_COARSEST, ST_VEC, ST_SCAL, ST_CHECK };

struct Stage {
    int kind = 0;
    int mode = 0;        // column-pass mode (fine) or scalar op
    void* dargs = nullptr;
    int* dfirst = nullptr;
    int nsys = 0;        // systems taking part (their sc pointers at dsc)
    DevScalars** dsc = nullptr;
    int total = 0;       // CTAs
    bool fp32 = false;
};

}  // namespace pbm

using namespace pbm;

struct pbm_batch {
    int device = 0;
    int nsys = 0;
    bool op_s = false;
    bool mixed = false;
    std::vector<pbm_grid*> g;
    std::vector<void*> allocs;            // device memory owned by the batch
    DevScalars** d_sc_all = nullptr;      // every system's scalar block
    double* d_ctl_in = nullptr;           // 3 per system
    double* d_gather = nullptr;           // GATHER per system
    double* h_pinned = nullptr;           // host mirror: ctl input then gather output
    // stage lists per vector precision p (0 FP64, 1 FP32)
    std::vector<Stage> init[2], iter[2], resid[2];
    cudaGraphExec_t graph[2] = {};
    int64_t graph_kernels[2] = {};
    cudaStream_t cap = nullptr;
};

namespace pbm {

static void* balloc(pbm_batch* b, size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
        (void)cudaGetLastError();
        fail(PBM_ENOMEM, "cudaMalloc failed for a batch table");
    }
    b->allocs.push_back(p);
    return p;
}

template <class A>
static Stage make_stage(pbm_batch* b, int kind, int mode, bool fp32, const std::vector<int>& sys,
                        const std::vector<A>& args, const std::vector<int>& blocks) {
    Stage st;
    st.kind = kind;
    st.mode = mode;
    st.fp32 = fp32;
    st.nsys = int(sys.size());
    std::vector<int> first(sys.size() + 1, 0);
    for (size_t i = 0; i < sys.size(); ++i) first[i + 1] = first[i] + blocks[i];
    st.total = first.back();
    std::vector<DevScalars*> sc(sys.size());
    for (size_t i = 0; i < sys.size(); ++i) sc[i] = b->g[sys[i]]->sc;
    st.dargs = balloc(b, sizeof(A) * args.size());
    st.dfirst = (int*)balloc(b, sizeof(int) * first.size());
    st.dsc = (DevScalars**)balloc(b, sizeof(DevScalars*) * sc.size());
    PBM_CUDA(cudaMemcpy(st.dargs, args.data(), sizeof(A) * args.size(), cudaMemcpyHostToDevice));
    PBM_CUDA(cudaMemcpy(st.dfirst, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
    PBM_CUDA(cudaMemcpy(st.dsc, sc.data(), sizeof(DevScalars*) * sc.size(), cudaMemcpyHostToDevice));
    return st;
}

static Stage make_scal_stage(pbm_batch* b, int op) {
    Stage st;
    st.kind = ST_SCAL;
    st.mode = op;
    st.nsys = b->nsys;
    st.dsc = b->d_sc_all;
    return st;
}

static void run_stage(const Stage& s, cudaStream_t st, cudaGraphConditionalHandle h = 0) {
    if (s.kind == ST_SCAL) {
        launch_scal_b(s.dsc, s.nsys, s.mode, st);
        return;
    }
    if (s.kind == ST_CHECK) {
        k_batch_check<<<1, 256, 0, st>>>(s.dsc, s.nsys, h);
        PBM_LAUNCH("batched check");
        return;
    }
    if (s.nsys == 0 || s.total == 0) return;
    const BatchMap M{s.dfirst, s.dsc, s.nsys};
    switch (s.kind) {
        case ST_FINE:
            if (s.fp32) launch_cols_fine_b<float>((const ColArgs<float>*)s.dargs, M, s.mode, s.total, st);
            else launch_cols_fine_b<double>((const ColArgs<double>*)s.dargs, M, s.mode, s.total, st);
            break;
        case ST_COARSE:
            if (s.fp32) launch_cols_coarse_b<float>((const ColArgs<float>*)s.dargs, M, s.total, st);
            else launch_cols_coarse_b<double>((const ColArgs<double>*)s.dargs, M, s.total, st);
            break;
        case ST_NODES:
            if (s.fp32) launch_nodes_b<float>((const NodeArgs<float>*)s.dargs, M, s.total, st);
            else launch_nodes_b<double>((const NodeArgs<double>*)s.dargs, M, s.total, st);
            break;
        case ST_RESTRICT:
            if (s.fp32) launch_restrict_b<float>((const RestrictArgs<float>*)s.dargs, M, s.total, st);
            else launch_restrict_b<double>((const RestrictArgs<double>*)s.dargs, M, s.total, st);
            break;
        case ST_PROLONG:
            if (s.fp32) launch_prolong_b<float>((const ProlongArgs<float>*)s.dargs, M, s.total, st);
            else launch_prolong_b<double>((const ProlongArgs<double>*)s.dargs, M, s.total, st);
            break;
        case ST_COARSEST:
            if (s.fp32) launch_coarsest_b<float>((const CoarsestArgs<float>*)s.dargs, M, s.total, st);
            else launch_coarsest_b<double>((const CoarsestArgs<double>*)s.dargs, M, s.total, st);
            break;
        default:  // ST_VEC
            if (s.fp32) launch_vec_b<float>((const VecArgs<float>*)s.dargs, M, s.total, st);
            else launch_vec_b<double>((const VecArgs<double>*)s.dargs, M, s.total, st);
            break;
    }
}

// ---- stage generation ---------------------------------------------------------------------------
template <class T>
struct Gen {
    pbm_batch* b;
    bool fp32;
    bool op_s;
    std::vector<Stage>* out;

    static int vec_blocks(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 608))); }
    int64_t nvec(int s, int k) const { return b->g[s]->L[k].g.n() + (op_s ? 1 : 0); }
    T* lv(int s, int k, char which) const {
        Level& L = b->g[s]->L[k];
        if (fp32) {
            switch (which) {
                case 't': return (T*)(void*)L.t32;
                case 'r': return (T*)(void*)L.r32;
                case 'x': return (T*)(void*)L.x32;
                case 'd': return (T*)(void*)L.idiag32;
                default: return (T*)(void*)L.b32;
            }
        }
        switch (which) {
            case 't': return (T*)(void*)L.t64;
            case 'r': return (T*)(void*)L.r64;
            case 'x': return (T*)(void*)L.x64;
            case 'd': return (T*)(void*)L.idiag64;
            default: return (T*)(void*)L.b64;
        }
    }
    T* pool(int s, int i) const {
        return fp32 ? (T*)(void*)b->g[s]->kv32[i] : (T*)(void*)b->g[s]->kv64[i];
    }

    // y = A x (+ epilogue) on level k of systems `sys`
    void apply(int k, const std::vector<int>& sys, const std::vector<ApplyArgs>& a) {
        if (sys.empty()) return;
        std::vector<ColArgs<T>> ca(sys.size());
        std::vector<NodeArgs<T>> na(sys.size());
        std::vector<int> cb(sys.size()), nb(sys.size());
        int mode = 0;
        for (size_t i = 0; i < sys.size(); ++i) {
            pbm_grid* g = b->g[sys[i]];
            ColEnv env = env_of(g);
            const Geom& G = g->L[k].g;
            ApplyArgs ai = a[i];
            ai.with_alpha = op_s;
            if (k == 0) {
                env.L = fine_L(g, fp32, op_s);
                const T* w = op_s ? (fp32 ? (const T*)(const void*)g->w32 : (const T*)(const void*)g->w64)
                                  : (fp32 ? (const T*)(const void*)g->rho32 : (const T*)(const void*)g->rho);
                const T* d = op_s ? (fp32 ? (const T*)(const void*)g->d32 : (const T*)(const void*)g->d64) : nullptr;
                const T* what = (op_s && !fp32) ? (const T*)(const void*)g->what_hat : nullptr;
                const T* u = (op_s && fp32) ? (const T*)(const void*)g->u32 : nullptr;
                ca[i] = make_fine_args<T>(env, G, g->kehat, w, d, what, u, ai.x, &cb[i]);
                mode = op_s ? (fp32 ? 2 : 1) : 0;
                na[i] = make_node_args<T>(env, G, ai, ca[i].L, (const T*)nullptr, nullptr,
                                          op_s ? g->partials : nullptr, op_s ? cb[i] : 0, op_s ? cb[i] : 0, &nb[i]);
            } else {
                const T* A = fp32 ? (const T*)(const void*)g->L[k].A32 : (const T*)(const void*)g->L[k].A64;
                const T* bord = fp32 ? (const T*)(const void*)g->L[k].bord32 : (const T*)(const void*)g->L[k].bord64;
                ca[i] = make_coarse_args<T>(env, G, A, ai.x, &cb[i]);
                na[i] = make_node_args<T>(env, G, ai, 1, bord, &g->sc->salpha, nullptr, 0, 0, &nb[i]);
            }
        }
        out->push_back(make_stage(b, k == 0 ? ST_FINE : ST_COARSE, mode, fp32, sys, ca, cb));
        out->push_back(make_stage(b, ST_NODES, 0, fp32, sys, na, nb));
    }

    void vec(const std::vector<int>& sys, const std::vector<VecArgs<T>>& va) {
        if (sys.empty()) return;
        std::vector<int> blocks(sys.size());
        for (size_t i = 0; i < sys.size(); ++i) blocks[i] = vec_blocks(va[i].n);
        out->push_back(make_stage(b, ST_VEC, 0, fp32, sys, va, blocks));
    }

    // x = M^{-1} b on level k for the systems `sys` (in[i] = b, outp[i] = x), dot x . b into red[dot_slot]
    // when dot_slot >= 0; first_done: the caller wrote the first smoothing sweep
    void vcycle(int k, const std::vector<int>& sys, const std::vector<const T*>& in, const std::vector<T*>& outp,
                int dot_slot, bool first_done) {
        std::vector<int> sc, ss;
        std::vector<size_t> ic, is;
        for (size_t i = 0; i < sys.size(); ++i) {
            if (k == b->g[sys[i]]->levels - 1) {
                sc.push_back(sys[i]);
                ic.push_back(i);
            } else {
                ss.push_back(sys[i]);
                is.push_back(i);
            }
        }
        if (!sc.empty()) {
            std::vector<CoarsestArgs<T>> ca(sc.size());
            std::vector<int> cb(sc.size());
            for (size_t j = 0; j < sc.size(); ++j)
                ca[j] = make_coarsest_args<T>(b->g[sc[j]], in[ic[j]], outp[ic[j]], op_s, &cb[j]);
            out->push_back(make_stage(b, ST_COARSEST, 0, fp32, sc, ca, cb));
        }
        if (ss.empty()) return;
        const int pre = b->g[ss[0]]->desc.pre_sweeps, post = b->g[ss[0]]->desc.post_sweeps;
        std::vector<T*> cur(ss.size()), oth(ss.size());
        for (size_t j = 0; j < ss.size(); ++j) {
            T* x = outp[is[j]];
            T* t = lv(ss[j], k, 't');
            cur[j] = (pre % 2 == 1) ? x : t;
            oth[j] = (cur[j] == x) ? t : x;
        }
        auto om = [&](int s) { return (const double*)&b->g[s]->sc->mr[16 + k]; };
        // Chebyshev smoothing (the batch's grids share the smoother): step sw >= 1 of a pass is EPI_CHEB
        const bool cheb = b->g[ss[0]]->desc.smoother == PBM_SMOOTHER_CHEBYSHEV;
        auto coef = [&](int s, int sw, bool pre_pass) {
            return (cheb && sw >= 1) ? (const double*)&b->g[s]->sc->cheb[k][cheb_slot(sw, pre_pass && sw == 1)] : om(s);
        };
        const int mode_cheb = EPI_CHEB;
        if (pre >= 1) {
            if (!first_done) {
                std::vector<VecArgs<T>> va(ss.size());
                for (size_t j = 0; j < ss.size(); ++j) {
                    VecArgs<T> v{};
                    v.op = VOP_FIRST_JACOBI;
                    v.n = nvec(ss[j], k);
                    v.a = in[is[j]];
                    v.f = lv(ss[j], k, 'd');
                    v.om = om(ss[j]);
                    v.b = cur[j];
                    va[j] = v;
                }
                vec(ss, va);
            }
            for (int sw = 1; sw < pre; ++sw) {
                std::vector<ApplyArgs> aa(ss.size());
                for (size_t j = 0; j < ss.size(); ++j) {
                    ApplyArgs a{};
                    a.x = cur[j];
                    a.y = oth[j];
                    a.b = in[is[j]];
                    a.diag = lv(ss[j], k, 'd');
                    a.omega = coef(ss[j], sw, true);
                    a.mode = cheb ? mode_cheb : EPI_JACOBI;
                    a.dot_slot = -1;
                    aa[j] = a;
                }
                apply(k, ss, aa);
                std::swap(cur, oth);
            }
        } else {
            fail(PBM_EINVAL, "batched V-cycle needs at least one pre-smoothing sweep");
        }
        // residual, restriction (with the next level's first sweep when it is not the coarsest)
        {
            std::vector<ApplyArgs> aa(ss.size());
            for (size_t j = 0; j < ss.size(); ++j) {
                ApplyArgs a{};
                a.x = outp[is[j]];
                a.y = lv(ss[j], k, 'r');
                a.b = in[is[j]];
                a.mode = EPI_RESID;
                a.dot_slot = -1;
                aa[j] = a;
            }
            apply(k, ss, aa);
        }
        std::vector<const T*> cin(ss.size());
        std::vector<T*> cout_(ss.size());
        std::vector<RestrictArgs<T>> ra(ss.size());
        std::vector<int> rb(ss.size());
        for (size_t j = 0; j < ss.size(); ++j) {
            pbm_grid* g = b->g[ss[j]];
            const bool fuse = (k + 1 < g->levels - 1);
            T* xc = lv(ss[j], k + 1, 'x');
            T* xfirst = fuse ? ((pre % 2 == 1) ? xc : lv(ss[j], k + 1, 't')) : nullptr;
            cin[j] = lv(ss[j], k + 1, 'b');
            cout_[j] = xc;
            ra[j] = make_restrict_args<T>(g, k, lv(ss[j], k, 'r'), lv(ss[j], k + 1, 'b'), op_s, 1.0, xfirst, &rb[j]);
        }
        out->push_back(make_stage(b, ST_RESTRICT, 0, fp32, ss, ra, rb));
        vcycle(k + 1, ss, cin, cout_, -1, true);
        {
            std::vector<ProlongArgs<T>> pa(ss.size());
            std::vector<int> pb(ss.size());
            for (size_t j = 0; j < ss.size(); ++j)
                pa[j] = make_prolong_args<T>(b->g[ss[j]], k, cout_[j], outp[is[j]], op_s, &pb[j]);
            out->push_back(make_stage(b, ST_PROLONG, 0, fp32, ss, pa, pb));
        }
        for (size_t j = 0; j < ss.size(); ++j) {
            cur[j] = outp[is[j]];
            oth[j] = lv(ss[j], k, 't');
        }
        for (int sw = 0; sw < post; ++sw) {
            std::vector<ApplyArgs> aa(ss.size());
            for (size_t j = 0; j < ss.size(); ++j) {
                ApplyArgs a{};
                a.x = cur[j];
                a.y = oth[j];
                a.b = in[is[j]];
                a.diag = lv(ss[j], k, 'd');
                a.omega = coef(ss[j], sw, false);
                a.mode = (cheb && sw >= 1) ? mode_cheb : EPI_JACOBI;
                a.dot_slot = (sw == post - 1) ? dot_slot : -1;
                aa[j] = a;
            }
            apply(k, ss, aa);
            std::swap(cur, oth);
        }
        if (post % 2 == 1) {
            std::vector<VecArgs<T>> va(ss.size());
            for (size_t j = 0; j < ss.size(); ++j) {
                VecArgs<T> v{};
                v.op = VOP_COPY;
                v.n = nvec(ss[j], k);
                v.a = cur[j];
                v.b = outp[is[j]];
                va[j] = v;
            }
            vec(ss, va);
        }
    }
};

// builds the stage lists of vector precision p (buffers: pool 0..6 MINRES, 10 iterate X, 11 rhs B)
template <class T>
static void build_plan(pbm_batch* b, int p) {
    const bool fp32 = p == 1;
    std::vector<int> all(b->nsys);
    for (int s = 0; s < b->nsys; ++s) all[s] = s;
    auto P = [&](int s, int i) { return fp32 ? (T*)(void*)b->g[s]->kv32[i] : (T*)(void*)b->g[s]->kv64[i]; };
    auto nv = [&](int s) { return b->g[s]->L[0].g.n() + (b->op_s ? 1 : 0); };
    auto apply0 = [&](Gen<T>& gen, int xi, int yi, int mode, int slot) {
        std::vector<ApplyArgs> aa(b->nsys);
        for (int s = 0; s < b->nsys; ++s) {
            ApplyArgs a{};
            a.x = P(s, xi);
            a.y = P(s, yi);
            a.b = P(s, 11);
            a.mode = mode;
            a.dot_slot = slot;
            aa[s] = a;
        }
        gen.apply(0, all, aa);
    };
    auto vecop = [&](Gen<T>& gen, int op, int ai, int bi, int ci, int di, int ei) {
        std::vector<VecArgs<T>> va(b->nsys);
        for (int s = 0; s < b->nsys; ++s) {
            VecArgs<T> v{};
            v.op = op;
            v.n = nv(s);
            v.a = ai >= 0 ? P(s, ai) : nullptr;
            v.b = bi >= 0 ? P(s, bi) : nullptr;
            v.c = ci >= 0 ? P(s, ci) : nullptr;
            v.d = di >= 0 ? P(s, di) : nullptr;
            v.e = ei >= 0 ? P(s, ei) : nullptr;
            v.mr = b->g[s]->sc->mr;
            v.red = b->g[s]->sc->red;
            va[s] = v;
        }
        gen.vec(all, va);
    };
    auto precond = [&](Gen<T>& gen, int in, int out) {
        std::vector<const T*> bi(b->nsys);
        std::vector<T*> xo(b->nsys);
        for (int s = 0; s < b->nsys; ++s) {
            bi[s] = P(s, in);
            xo[s] = P(s, out);
        }
        gen.vcycle(0, all, bi, xo, 1, false);
    };
    // init: r = B - A X -> V1 (red[2]), Zc = M^-1 V1 (red[1]), MINRES start, V0 = D1 = D2 = 0
    {
        Gen<T> gen{b, fp32, b->op_s, &b->init[p]};
        apply0(gen, 10, 1, EPI_RESID, 2);
        precond(gen, 1, 2);
        b->init[p].push_back(make_scal_stage(b, SOP_INIT));
        vecop(gen, VOP_ZERO, -1, 0, -1, -1, -1);
        vecop(gen, VOP_ZERO, -1, 4, -1, -1, -1);
        vecop(gen, VOP_ZERO, -1, 5, -1, -1, -1);
    }
    // iteration: AZ = A Zc (red[0]); Lanczos; Zn = M^-1 V1 (red[1]); Givens; update; check
    {
        Gen<T> gen{b, fp32, b->op_s, &b->iter[p]};
        apply0(gen, 2, 6, EPI_APPLY, 0);
        vecop(gen, VOP_LANCZOS2, 6, 0, 1, -1, -1);
        precond(gen, 1, 3);
        b->iter[p].push_back(make_scal_stage(b, SOP_SCALARS));
        vecop(gen, VOP_UPDATE2, 3, 2, 4, 5, 10);
        Stage chk;
        chk.kind = ST_CHECK;
        chk.nsys = b->nsys;
        chk.dsc = b->d_sc_all;
        b->iter[p].push_back(chk);
    }
    // true residual: r = B - A X -> AZ (red[2])
    {
        Gen<T> gen{b, fp32, b->op_s, &b->resid[p]};
        apply0(gen, 10, 6, EPI_RESID, 2);
    }
}

static cudaGraphExec_t batch_graph(pbm_batch* b, int p) {
    if (b->graph[p]) return b->graph[p];
    if (!b->cap) PBM_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
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
        PBM_CUDA(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        try {
            for (const Stage& s : b->iter[p]) run_stage(s, b->cap, h);
        } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(b->cap, &dummy);
            throw;
        }
        PBM_CUDA(cudaStreamEndCapture(b->cap, &body));
        PBM_CUDA(cudaGraphInstantiate(&b->graph[p], graph, 0));
    } catch (...) {
        cudaGraphDestroy(graph);
        count_launch_add(before - launch_count());
        throw;
    }
    cudaGraphDestroy(graph);
    b->graph_kernels[p] = launch_count() - before;
    count_launch_add(-b->graph_kernels[p]);
    return b->graph[p];
}

// host side of one round of batched MINRES on precision p: per system rhs in pool 11, iterate in
// pool 10 (already in place), rtol per system; `active` in: systems to solve, out: unchanged.
// Returns per-system (status, iterations, relres).
struct SysResult {
    int status = PBM_OK;
    int iters = 0;
    double relres = 0.0;
};

static void set_ctl(pbm_batch* b, const std::vector<double>& target, const std::vector<int>& budget,
                    const std::vector<int>& active, cudaStream_t st) {
    for (int s = 0; s < b->nsys; ++s) {
        b->h_pinned[3 * s] = target[s];
        b->h_pinned[3 * s + 1] = double(budget[s]);
        b->h_pinned[3 * s + 2] = active[s] ? 1.0 : 0.0;
    }
    PBM_CUDA(cudaMemcpyAsync(b->d_ctl_in, b->h_pinned, sizeof(double) * 3 * b->nsys, cudaMemcpyHostToDevice, st));
    k_batch_ctl<<<(b->nsys + 63) / 64, 64, 0, st>>>(b->d_sc_all, b->nsys, b->d_ctl_in);
    PBM_LAUNCH("batched control");
    // the pinned buffer is reused for the gather: finish the upload first
    PBM_CUDA(cudaStreamSynchronize(st));
}

static const double* gather(pbm_batch* b, cudaStream_t st) {
    k_batch_gather<<<(b->nsys + 63) / 64, 64, 0, st>>>(b->d_sc_all, b->nsys, b->d_gather);
    PBM_LAUNCH("batched gather");
    PBM_CUDA(cudaMemcpyAsync(b->h_pinned, b->d_gather, sizeof(double) * GATHER * b->nsys, cudaMemcpyDeviceToHost,
                             st));
    PBM_CUDA(cudaStreamSynchronize(st));
    return b->h_pinned;
}

static std::vector<SysResult> batch_minres(pbm_batch* b, int p, const std::vector<double>& rtol,
                                           std::vector<int> active, int maxit, bool check_true, cudaStream_t st) {
    const int ns = b->nsys;
    std::vector<SysResult> res(ns);
    // |B|^2 per system (red[3])
    for (int s = 0; s < ns; ++s) {
        if (!active[s]) continue;
        pbm_grid* g = b->g[s];
        const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
        const void* B = p ? (const void*)g->kv32[11] : (const void*)g->kv64[11];
        launch_dot(g, p == 1, B, B, nv, 3, st);
    }
    std::vector<double> bnorm(ns, 0.0), target(rtol), last(ns, std::numeric_limits<double>::infinity());
    {
        const double* G = gather(b, st);
        for (int s = 0; s < ns; ++s) {
            bnorm[s] = std::sqrt(G[GATHER * s + 6]);
            if (active[s] && bnorm[s] == 0.0) active[s] = 0;   // zero right-hand side: x stays as given
        }
    }
    std::vector<int> budget(ns, maxit);
    set_ctl(b, target, budget, active, st);
    for (const Stage& s : b->init[p]) run_stage(s, st);
    {
        const double* G = gather(b, st);
        for (int s = 0; s < ns; ++s)
            if (active[s] && G[GATHER * s + 4] != 0.0) {
                res[s].status = PBM_EBREAKDOWN;
                active[s] = 0;
            }
    }
    const bool graph = true;
    while (true) {
        bool any = false;
        for (int s = 0; s < ns; ++s) {
            budget[s] = maxit - res[s].iters;
            if (active[s] && budget[s] <= 0) {
                res[s].status = PBM_ENOTCONV;
                active[s] = 0;
            }
            any = any || active[s];
        }
        if (!any) break;
        set_ctl(b, target, budget, active, st);
        if (graph) {
            cudaGraphExec_t ex = batch_graph(b, p);
            PBM_CUDA(cudaGraphLaunch(ex, st));
        }
        const double* G = gather(b, st);
        std::vector<int> check(ns, 0);
        bool any_check = false;
        int64_t iters_run = 0;
        for (int s = 0; s < ns; ++s) {
            if (!active[s]) continue;
            const int it = int(G[GATHER * s]);
            iters_run = std::max<int64_t>(iters_run, it);
            res[s].iters += it;
            const int reason = int(G[GATHER * s + 1]);
            if (reason == 1) {
                res[s].status = PBM_EBREAKDOWN;
                active[s] = 0;
            } else if (reason == 2 || reason == 3) {
                if (!check_true) {
                    active[s] = 0;
                } else {
                    check[s] = 1 + (reason == 2 ? 1 : 0);
                    any_check = true;
                }
            } else if (reason == 4) {
                res[s].status = PBM_ENOTCONV;
                active[s] = 0;
            }
        }
        count_launch_add(b->graph_kernels[p] * iters_run);
        if (!any_check) continue;
        // true residuals of the systems whose estimate reached its target
        std::vector<int> act2(ns, 0);
        for (int s = 0; s < ns; ++s) act2[s] = check[s] ? 1 : 0;
        set_ctl(b, target, budget, act2, st);
        for (const Stage& s : b->resid[p]) run_stage(s, st);
        G = gather(b, st);
        for (int s = 0; s < ns; ++s) {
            if (!check[s]) continue;
            const double rel = std::sqrt(G[GATHER * s + 5]) / bnorm[s];
            res[s].relres = rel;
            if (rel <= rtol[s]) {
                active[s] = 0;
            } else if (check[s] == 2 || !(rel < 0.5 * last[s])) {
                res[s].status = PBM_ENOTCONV;
                active[s] = 0;
            } else {
                last[s] = rel;
                target[s] = target[s] * 0.5 * rtol[s] / rel;
            }
        }
    }
    return res;
}

}  // namespace pbm

extern "C" {

int pbm_batch_create(pbm_grid* const* grids, int n, int op, pbm_batch** out) {
    pbm_batch* b = nullptr;
    try {
        if (!grids || !out || n < 1) fail(PBM_EINVAL, "null argument or empty batch");
        if (op != PBM_OP_K && op != PBM_OP_S) fail(PBM_EINVAL, "unknown operator");
        *out = nullptr;
        b = new pbm_batch();
        b->nsys = n;
        b->op_s = op == PBM_OP_S;
        b->g.assign(grids, grids + n);
        b->device = grids[0]->device;
        b->mixed = grids[0]->desc.precision == PBM_MIXED;
        for (int s = 0; s < n; ++s) {
            pbm_grid* g = grids[s];
            if (!g) fail(PBM_EINVAL, "null grid in the batch");
            if (g->device != b->device) fail(PBM_EINVAL, "all grids of a batch must live on one device");
            if ((g->desc.precision == PBM_MIXED) != b->mixed) fail(PBM_EINVAL, "all grids of a batch need one precision");
            if (g->desc.pre_sweeps < 1) fail(PBM_EINVAL, "batched V-cycles need at least one pre-smoothing sweep");
            if (g->desc.smoother == PBM_SMOOTHER_GAUSS_SEIDEL)
                fail(PBM_EINVAL, "batched V-cycles smooth with Jacobi or Chebyshev, not Gauss-Seidel");
            if (g->desc.pre_sweeps != grids[0]->desc.pre_sweeps || g->desc.post_sweeps != grids[0]->desc.post_sweeps ||
                g->desc.smoother != grids[0]->desc.smoother)
                fail(PBM_EINVAL, "all grids of a batch need the same smoothing sweeps");
            if (g->prof_on) fail(PBM_EINVAL, "profiling must be off for batched solves");
            for (int t = 0; t < s; ++t)
                if (grids[t] == g) fail(PBM_EINVAL, "a grid appears twice in the batch");
        }
        PBM_CUDA(cudaSetDevice(b->device));
        std::vector<DevScalars*> sc(n);
        for (int s = 0; s < n; ++s) sc[s] = grids[s]->sc;
        b->d_sc_all = (DevScalars**)balloc(b, sizeof(DevScalars*) * n);
        PBM_CUDA(cudaMemcpy(b->d_sc_all, sc.data(), sizeof(DevScalars*) * n, cudaMemcpyHostToDevice));
        b->d_ctl_in = (double*)balloc(b, sizeof(double) * 3 * n);
        b->d_gather = (double*)balloc(b, sizeof(double) * GATHER * n);
        PBM_CUDA(cudaMallocHost((void**)&b->h_pinned, sizeof(double) * (GATHER + 3) * n));
        build_plan<double>(b, 0);
        if (b->mixed) build_plan<float>(b, 1);
        *out = b;
        b = nullptr;
    } catch (const Error& e) {
        set_error(e.msg);
        if (b) pbm_batch_destroy(b);
        return e.code;
    }
    set_error("");
    return PBM_OK;
}

int pbm_batch_destroy(pbm_batch* b) {
    if (!b) return PBM_OK;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    for (cudaGraphExec_t e : b->graph)
        if (e) cudaGraphExecDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_pinned) cudaFreeHost(b->h_pinned);
    delete b;
    return PBM_OK;
}

int pbm_batch_minres_solve(pbm_batch* b, const double* const* b_dev, double* const* x_dev, double rtol, int maxit,
                           pbm_solve_info* infos, void* stream) {
    try {
        if (!b || !b_dev || !x_dev) fail(PBM_EINVAL, "null argument");
        if (!(rtol > 0.0) || maxit < 1) fail(PBM_EINVAL, "rtol must be > 0 and maxit >= 1");
        PBM_CUDA(cudaSetDevice(b->device));
        const cudaStream_t st = (cudaStream_t)stream;
        const int ns = b->nsys;
        auto t0 = std::chrono::steady_clock::now();
        for (int s = 0; s < ns; ++s) {
            pbm_grid* g = b->g[s];
            if (!b_dev[s] || !x_dev[s]) fail(PBM_EINVAL, "null vector in the batch");
            const int need = b->op_s ? 2 : 1;
            if (b->op_s ? !g->state_set : !g->rho_set) fail(PBM_ESTATE, "operator of a batch system is not set");
            if (g->op_ready != need) fail(PBM_ESTATE, "hierarchy of a batch system is not current (set-up first)");
        }
        std::vector<pbm_solve_info> inf(ns);
        std::vector<int> active(ns, 1);
        if (!b->mixed) {
            for (int s = 0; s < ns; ++s) {
                pbm_grid* g = b->g[s];
                const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                PBM_CUDA(cudaMemcpyAsync(g->kv64[11], b_dev[s], sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
                PBM_CUDA(cudaMemcpyAsync(g->kv64[10], x_dev[s], sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
            }
            std::vector<double> tol(ns, rtol);
            std::vector<SysResult> r = batch_minres(b, 0, tol, active, maxit, true, st);
            for (int s = 0; s < ns; ++s) {
                pbm_grid* g = b->g[s];
                const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                PBM_CUDA(cudaMemcpyAsync(x_dev[s], g->kv64[10], sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
                inf[s].status = r[s].status;
                inf[s].iterations = r[s].iters;
                inf[s].outer = 1;
                inf[s].relres = r[s].relres;
            }
        } else {
            // FP64 iterative refinement around batched FP32 inner solves; a system whose step does
            // not halve the FP64 residual finishes with the single-system robust stage
            std::vector<double> rel(ns, 0.0), bn(ns, 0.0);
            std::vector<int> robust(ns, 0), total(ns, 0), outer(ns, 0);
            for (int s = 0; s < ns; ++s) {
                pbm_grid* g = b->g[s];
                const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                PBM_CUDA(cudaMemcpyAsync(g->kv64[11], b_dev[s], sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
                PBM_CUDA(cudaMemcpyAsync(g->kv64[10], x_dev[s], sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
                launch_dot(g, false, g->kv64[11], g->kv64[11], nv, 3, st);
            }
            {
                const double* G = gather(b, st);
                for (int s = 0; s < ns; ++s) bn[s] = std::sqrt(G[GATHER * s + 6]);
            }
            auto fp64_resid = [&](const std::vector<int>& act) {
                set_ctl(b, std::vector<double>(ns, 0.0), std::vector<int>(ns, 0), act, st);
                for (const Stage& sg : b->resid[0]) run_stage(sg, st);
                const double* G = gather(b, st);
                for (int s = 0; s < ns; ++s)
                    if (act[s]) rel[s] = bn[s] > 0.0 ? std::sqrt(G[GATHER * s + 5]) / bn[s] : 0.0;
            };
            fp64_resid(active);
            for (int s = 0; s < ns; ++s)
                if (rel[s] <= rtol) active[s] = 0;
            for (int step = 0; step < 60; ++step) {
                bool any = false;
                for (int s = 0; s < ns; ++s) any = any || active[s];
                if (!any) break;
                // inner rhs: the FP64 residual (pool 6 after the residual stage) rounded to FP32
                for (int s = 0; s < ns; ++s) {
                    if (!active[s]) continue;
                    pbm_grid* g = b->g[s];
                    const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                    launch_cast(g->kv64[6], false, g->kv32[11], true, nv, st);
                    PBM_CUDA(cudaMemsetAsync(g->kv32[10], 0, sizeof(float) * nv, st));
                    outer[s] += 1;
                }
                std::vector<double> itol(ns, b->g[0]->desc.inner_rtol);
                std::vector<int> budget_left(ns, 0);
                int mx = 1;
                for (int s = 0; s < ns; ++s) mx = std::max(mx, maxit - total[s]);
                std::vector<SysResult> r = batch_minres(b, 1, itol, active, mx, false, st);
                std::vector<double> prev(rel);
                for (int s = 0; s < ns; ++s) {
                    if (!active[s]) continue;
                    total[s] += r[s].iters;
                    pbm_grid* g = b->g[s];
                    const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                    if (r[s].status == PBM_EBREAKDOWN) {
                        robust[s] = 1;
                        active[s] = 0;
                        continue;
                    }
                    add_f32(g->kv64[10], g->kv32[10], nv, st, 1.0);
                }
                std::vector<int> act(active);
                fp64_resid(act);
                for (int s = 0; s < ns; ++s) {
                    if (!active[s]) continue;
                    pbm_grid* g = b->g[s];
                    const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                    if (rel[s] <= rtol) {
                        active[s] = 0;
                    } else if (!(rel[s] < 0.5 * prev[s])) {
                        if (!(rel[s] < prev[s])) {
                            add_f32(g->kv64[10], g->kv32[10], nv, st, -1.0);
                            rel[s] = prev[s];
                        }
                        robust[s] = 1;
                        active[s] = 0;
                    } else if (total[s] >= maxit) {
                        active[s] = 0;
                    }
                }
            }
            for (int s = 0; s < ns; ++s) {
                pbm_grid* g = b->g[s];
                const int64_t nv = g->L[0].g.n() + (b->op_s ? 1 : 0);
                PBM_CUDA(cudaMemcpyAsync(x_dev[s], g->kv64[10], sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
                inf[s].iterations = total[s];
                inf[s].outer = outer[s];
                inf[s].relres = rel[s];
                inf[s].status = rel[s] <= rtol ? PBM_OK : PBM_ENOTCONV;
                if (robust[s] && rel[s] > rtol) {
                    pbm_solve_info si{};
                    solve(g, b->op_s, b_dev[s], x_dev[s], rtol, std::max(1, maxit - total[s]), &si, st);
                    inf[s].iterations += si.iterations;
                    inf[s].outer += si.outer;
                    inf[s].relres = si.relres;
                    inf[s].status = si.status;
                }
            }
        }
        PBM_CUDA(cudaStreamSynchronize(st));
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        int worst = PBM_OK;
        for (int s = 0; s < ns; ++s) {
            inf[s].solve_ms = ms;
            if (inf[s].status != PBM_OK && worst == PBM_OK) worst = inf[s].status;
            if (infos) infos[s] = inf[s];
        }
        if (worst != PBM_OK) {
            set_error("a system of the batch did not reach the tolerance");
            return worst;
        }
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    }
    set_error("");
    return PBM_OK;
}

}  // extern "C"
