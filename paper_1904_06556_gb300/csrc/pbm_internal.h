// Internal declarations of the reduced-Newton MG-MINRES library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "pbm.h"

namespace pbm {

// ------------------------------------------------------------------------------------------------
// error handling
// ------------------------------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};
void set_error(const std::string& msg);
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
void count_launch();  // process-wide counter of the kernels this library launched
void count_launch_add(int64_t delta);
int64_t launch_count();
// Number of SMs of the current device, queried once per device and cached. The launches whose CTA
// count is fixed (so that their reductions sum in a fixed order) and the wave models of the tile
// planners size themselves from it: results are bit-reproducible on a given device, and a part with
// another SM count is filled the same way.
int num_sms();
constexpr int kNodeBlocksPerSm = 8;   // CTA cap of the node pass of the two-pass operators, per SM
#define PBM_CUDA(x) ::pbm::check_cuda((x), #x)
#define PBM_LAUNCH(what) (::pbm::count_launch(), ::pbm::check_cuda(cudaGetLastError(), what))

// ------------------------------------------------------------------------------------------------
// programmatic dependent launch on the solve path: launch_pdl lets the launch of the next kernel of
// the stream overlap the end of this one; every kernel launched that way begins with pdl_wait() (its
// predecessor has completed and its writes are visible after it). Kernels of more than one CTA per SM
// do not trigger their successors early (pdl_launch): waiting CTAs of the next kernel would take
// registers and warp slots from the running one, which slowed the FP64 solve down by a quarter. In a
// kernel launched normally pdl_wait() is a no-op.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// The exception: a grid of at most one CTA per SM (the coarse levels, the transfers to them, the coarsest solve)
// lets the next kernel of the stream launch once its own predecessor has completed (call after pdl_wait()): the
// waiting CTAs of the next kernel sit on SMs this grid leaves idle, and the launch gaps of the V-cycle's chains
// of small kernels overlap the running kernel.
__device__ __forceinline__ void pdl_launch_if_small() {
    unsigned nsm;
    asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
    if (gridDim.x * gridDim.y * gridDim.z <= nsm) pdl_launch();
}

// Last-CTA completion of the ordered reductions: this thread's share a[t], a[t + stride], ... of the per-CTA
// partials a[0 .. n) summed in that order. The partials were written by other CTAs before their fence, so they are
// read from L2 (ld.global.cg); the loads are issued eight at a time, so a long share costs one L2 round trip per
// eight entries instead of one per entry, with the same additions in the same order.
__device__ __forceinline__ double l2_strided_sum(const double* a, int n, int t, int stride) {
    double s = 0.0;
    for (int q0 = t; q0 < n; q0 += 8 * stride) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * stride;
            v[u] = q < n ? __ldcg(a + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (q0 + u * stride < n) s += v[u];
    }
    return s;
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    check_cuda(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...), "kernel launch");
}

// ------------------------------------------------------------------------------------------------
// geometry of one level (structured grid of cubes)
// ------------------------------------------------------------------------------------------------
struct Geom {
    int nx, ny, nz;      // elements
    int support;         // enum pbm_support
    int64_t nnode() const { return int64_t(nx + 1) * (ny + 1) * (nz + 1); }
    int64_t n() const { return 3 * nnode(); }
    int64_t m() const { return int64_t(nx) * ny * nz; }
};

// Is node (i, j, k) of a level supported? The supports of the coarse levels are those of the same
// physical faces/corners/edges, so every level uses the same rule on its own node coordinates.
__host__ __device__ inline bool node_fixed(int support, int nx, int ny, int nz, int i, int j, int k) {
    (void)nz;
    switch (support) {
        case PBM_CANTILEVER: return i == 0;
        case PBM_BRIDGE_CORNERS: return k == 0 && (i == 0 || i == nx) && (j == 0 || j == ny);
        case PBM_BRIDGE_EDGES: return k == 0 && (i == 0 || i == nx);
        default: return false;
    }
}

// Support of node (i, j) as two bits: bit 0 fixed on planes k >= 1, bit 1 fixed on plane 0. Every
// support of node_fixed depends on the plane only through k == 0.
__host__ __device__ inline int fixed_bits(int support, int nx, int ny, int nz, int i, int j) {
    return (node_fixed(support, nx, ny, nz, i, j, 1) ? 1 : 0) | (node_fixed(support, nx, ny, nz, i, j, 0) ? 2 : 0);
}

// ------------------------------------------------------------------------------------------------
// element matrix of the fine level in the (sum, difference) tensor basis
//
// With H1 = [[1, 1], [-1, 1]] acting on the two nodal values along one direction and H = H1 (x) H1
// (x) H1 on the 8 nodal values of one displacement component, the Q1 element matrix factors as
//     K_e x = H^T Khat H x,
// because each 1D integral matrix (int N'N', int NN, int N'N, int NN') maps the sum / difference
// coefficients onto a single coefficient. Khat couples pattern q of output component c with at most
// three input coefficients:
//   diagonal:          dg[c][q] * X_c[q]
//   for d != c, r the third direction:
//     q_c = 1, q_d = 0:  lam4[q_r] * X_d[q with bit c cleared and bit d set]
//     q_d = 1, q_c = 0:  mu4[q_r]  * X_d[q with bit d cleared and bit c set]
// lam4[b] = h lambda m(b) / 4, mu4[b] = h mu m(b) / 4, m(0) = 1/4, m(1) = 1/12, and
// dg[c][q] = h [ (lambda + mu) q_c m(q_a) m(q_b) + mu sum_{k: q_k = 1} prod_{j != k} m(q_j) ].
// ------------------------------------------------------------------------------------------------
struct KeHat {
    double dg[3][8];
    double lam4[2];
    double mu4[2];
};

// the factors of the isotropic Q1 cube of edge h (capi.cu)
void element_hat(double E, double nu, double h, KeHat& K);

template <class T>
struct KeHatT {
    T dg[3][8];
    T lam4[2];
    T mu4[2];
};

// per-component forward transform X = H v (index bits: 0 = x, 1 = y, 2 = z)
template <class T>
__device__ __forceinline__ void wht_fwd(T* v) {
#pragma unroll
    for (int s = 1; s < 8; s <<= 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if ((i & s) == 0) {
                T a = v[i], b = v[i + s];
                v[i] = a + b;
                v[i + s] = b - a;
            }
        }
    }
}

// per-component output transform y = H^T Y
template <class T>
__device__ __forceinline__ void wht_out(T* v) {
#pragma unroll
    for (int s = 1; s < 8; s <<= 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if ((i & s) == 0) {
                T a = v[i], b = v[i + s];
                v[i] = a - b;
                v[i + s] = a + b;
            }
        }
    }
}

// Y = Khat X on transformed coefficients X[c][q]. The DC pattern q = 0 is zero on output and never
// read (rigid translations are in the kernel of K_e).
template <class T>
__device__ __forceinline__ void khat_apply(const KeHatT<T>& K, const T (&X)[3][8], T (&Y)[3][8]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Y[c][0] = T(0);
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            T acc = K.dg[c][q] * X[c][q];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d == c) continue;
                const int r = 3 - c - d;
                const int br = (q >> r) & 1;
                const int qc = (q >> c) & 1, qd = (q >> d) & 1;
                if (qc == 1 && qd == 0) acc += K.lam4[br] * X[d][(q & ~(1 << c)) | (1 << d)];
                if (qd == 1 && qc == 0) acc += K.mu4[br] * X[d][(q & ~(1 << d)) | (1 << c)];
            }
            Y[c][q] = acc;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// one multigrid level
// ------------------------------------------------------------------------------------------------
struct Level {
    Geom g;
    double h = 1.0;
    // coarse levels: element matrices, upper triangle (i <= j) of the 24 x 24 matrix, entry-major
    // (entry t of element e at [t * m + e]); index of (i, j) is tri_index(i, j)
    double* A64 = nullptr;
    float* A32 = nullptr;
    // alpha border of S on this level (n entries; b_0 = -sum_i d_i K_i u, b_{k+1} = P^T b_k)
    double* bord64 = nullptr;
    float* bord32 = nullptr;
    // Jacobi diagonal, its inverse and its inverse square root (Lanczos), n + 1 entries (last = alpha)
    double* diag64 = nullptr;
    double* idiag64 = nullptr;
    double* sdiag64 = nullptr;
    float* idiag32 = nullptr;
    // V-cycle work vectors, n + 1 entries each
    double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *t64 = nullptr;
    float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr, *t32 = nullptr;
    double omega = 0.0, lambda_max = 0.0;
    // coarse levels: plane-quad scratch of this level's two-pass applies (12 (nz + 1) nx ny entries of
    // the FP64 size each), so that different levels can be applied on concurrent streams
    void* qa = nullptr;
    void* qb = nullptr;
};

constexpr int NTRI = 300;  // entries of the upper triangle of a 24 x 24 matrix
__host__ __device__ inline int tri_index(int i, int j) {  // i <= j
    return i * 24 - (i * (i - 1)) / 2 + (j - i);
}

// the element matrix as the operand of the tensor-core kernel: hi and lo parts (2 x 1024 floats) of
// K_e / scale in the MMA layout, and the number of MMA terms (2 when K_e / scale is exact in TF32)
struct TcMatrix {
    const float* B = nullptr;
    int terms = 3;
    float scale = 1.0f;
};

// device scalar block used by the reductions, Lanczos and MINRES
struct DevScalars {
    double red[64];        // reduction outputs (slot per use)
    double lz_a[128], lz_b[128];   // Lanczos coefficients, steps x level
    double mr[32];         // MINRES scalar state
    unsigned int counter[64];  // last-block-done counters (one per reduction slot)
    int flags[8];
    double salpha;         // S_alpha,alpha = sum_i d_i of the current state (coarse S applies)
    double cheb[16][4 * 2 * 8];   // per level: Chebyshev step coefficients (c0, c1, c2, 0) at cheb_slot
    double ctl[8];         // graph-resident MINRES loop control: target, iteration budget, count, exit
};

}  // namespace pbm

// ------------------------------------------------------------------------------------------------
// the handle
// ------------------------------------------------------------------------------------------------
struct pbm_grid {
    pbm_grid_desc desc;
    int device = 0;
    int levels = 1;
    std::vector<pbm::Level> L;
    pbm::KeHat kehat;                 // fine level, h-scaled
    double Ke[576];                   // fine-level element matrix (row-major), FP64
    double Kdiag;                     // K_e[i][i] (all equal for the isotropic cube)
    double G[8][576];                 // P_c^T K_e P_c for the 8 children (coarse local dofs)
    double* G_dev = nullptr;          // 8 x NTRI upper triangles, [c][t]
    float* G32 = nullptr;             // the same rounded to FP32, for the FP32 Galerkin chain of mixed grids
    float* tcB = nullptr;             // element matrix as the tensor-core operand (2 x 1024 floats)
    pbm::TcMatrix tc;
    // fine-level element data
    double* rho = nullptr;            // density (m)
    double* w64 = nullptr;            // element weights of the current operator (rho or rho')
    double* d64 = nullptr;            // Schur weights d_i
    double* eps64 = nullptr;          // rhs weights eps_i
    double* aux64 = nullptr;          // 8 m: 5 coefficient rows (rho'', mu''_lo, mu''_up, dL/dnu_lo,
                                      // dL/dnu_up), u^T K_e u, u^T K_e du, du^T K_e du
    double* wr64 = nullptr;           // rho' - eps (rhs weights)
    float* rho32 = nullptr;
    float* w32 = nullptr;
    float* d32 = nullptr;
    double* u64 = nullptr;            // masked displacement of the Newton state (n)
    float* u32 = nullptr;
    double* what = nullptr;           // P_c^T (K_e u_e) for every fine element, [24][m]
    double* what_hat = nullptr;       // Khat H u_e for every fine element, [21][m] (FP64 S pass)
    void* qa = nullptr;               // plane-quad scratch of the column passes, 12 (nz + 1) nx ny
    void* qb = nullptr;               // chunk-top quads, 12 nz nx ny (entries of the FP64 size)
    double* nwt = nullptr;            // Newton step buffers: dz (n + 1), r (n), dnu_lo (m), dnu_up (m)
    double s_alpha = 0.0;             // S_alpha,alpha = sum_i d_i
    // coarsest level: dense inverse of the bordered matrix, (nc+1)^2 FP64
    int nc = 0;
    double* cinv = nullptr;
    double* cwork = nullptr;
    // reductions
    double* partials = nullptr;       // per-block partial sums
    int max_blocks = 0;
    pbm::DevScalars* sc = nullptr;
    pbm::DevScalars* sc_host = nullptr;  // pinned mirror
    // Krylov work vectors (n + 1 of the finest level); [10] holds the MINRES iterate
    double* kv64[12] = {};
    float* kv32[12] = {};
    // operator state: 0 = none, 1 = K(rho) hierarchy current, 2 = S hierarchy current
    int op_ready = 0;
    bool rho_set = false;
    bool state_set = false;           // a PBM state (pbm_set_state) defines S
    bool ip_set = false;              // an interior-point state (pbm_ip_set_state) defines S
    double ip_rho_lo = 0.0, ip_rho_up = 1.0;
    double* ip_work = nullptr;        // 2 (n + 1): interior-point right-hand side and operand copies
    double alpha = 0.0, V = 0.0;      // of the current state
    double sum_rho1 = 0.0, sum_wr = 0.0, gl2 = 0.0;   // reductions of the coefficient kernel
    int64_t bytes = 0;
    // optional timing of the fine-level operator kernel (pbm_profile): CUDA event pairs recorded on
    // the launch stream around every fine apply, folded into the totals when read
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;      // 2 per recorded launch
    size_t prof_used = 0;
    pbm_profile_stats prof[2] = {};        // [PBM_OP_K], [PBM_OP_S]
    // MINRES iterations captured as CUDA graphs (a WHILE node around one iteration), per
    // (vector precision, operator, FP32 preconditioner); built on first use, kept until destroy
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t mr_graph[8] = {};
    int fineL[2][2] = {};                  // autotuned chunk length [fp32][op_s] of the fine column pass
    int fusedP[2] = {};                    // autotuned tile plan [op_s] of the single-pass FP32 operator
    bool coarse64_ready = false;           // FP64 coarse matrices and diagonals current (mixed grids build
                                           // them on first use, ensure_coarse64)
    int coarseP[2][16] = {};               // autotuned FP32 coarse operator [op_s][level]: -1 two passes
                                           // (eight threads per element), -2 two passes (a thread per
                                           // element), >= 0 plan of the single pass
    int64_t mr_graph_kernels[8] = {};      // kernels in one iteration of each graph (launch counting)
    std::vector<int> prof_op;              // operator of every recorded launch
    // set-up streams: the coarsest factorisation and the Lanczos estimates of the coarse levels run
    // beside the fine level's (created on first use)
    cudaStream_t side[16] = {};
    cudaEvent_t side_ev[19] = {};          // [k]: level k's stream done, [16]: fork, [17]: Galerkin chain done,
                                           // [18]: fine-level border done
};

namespace pbm {

void* dalloc(pbm_grid* g, size_t bytes);
void dfree(void* p);

// ---- kernels (launch wrappers), apply.cu ----
// EPI_CHEB: one step of Chebyshev acceleration of Jacobi, y = c0 x - c1 y_prev + c2 D^{-1} (b - A x)
// with (c0, c1, c2) = (1 + a_s, a_s or 0, b_s) read from ApplyArgs::omega, y_prev the iterate before x,
// read from y itself before it is overwritten (not read when c1 = 0)
// EPI_GS0 + c (c = 0 .. 24): one colour step of a multicolour Gauss-Seidel sweep: y = x + D^{-1} (b - A x) on the
// dofs of colour c = 3 node_colour + component (c = 24: the alpha entry of S), y = x elsewhere; no two dofs of
// one colour are coupled, so a sweep is point Gauss-Seidel in the colour ordering
enum EpiMode { EPI_APPLY = 0, EPI_RESID = 1, EPI_JACOBI = 2, EPI_CHEB = 3, EPI_GS0 = 4 };
__host__ __device__ inline int node_colour(int i, int j, int k) { return (i & 1) | ((j & 1) << 1) | ((k & 1) << 2); }
constexpr int kGsColours = 24;   // dof colours; alpha is colour 24
// slot of step s >= 1 (from_zero: the step after a first step taken from x = 0) in DevScalars::cheb[k]
constexpr int kChebMaxStep = 8;
inline int cheb_slot(int s, bool from_zero) { return 4 * (2 * (s - 1) + (from_zero ? 1 : 0)); }

struct ApplyArgs {
    // input vector (n (+1)), output (n (+1)); b and diag for RESID / JACOBI
    const void* x;
    void* y;
    const void* b;
    const void* diag;
    const double* omega;   // device scalar (JACOBI)
    int mode;
    bool with_alpha;       // vectors carry the alpha entry (operator S)
    int dot_slot;          // >= 0: accumulate sum(y_out . x) (APPLY) or ||y_out||^2 (RESID) or
                           // sum(y_out . b) (JACOBI) into sc->red[dot_slot]
    int rset = 0;          // reduction set: launches that may run concurrently on different streams
                           // use different sets (partial sums and last-CTA counter, see red_set)
};

// Scratch of the cross-CTA reductions of one launch: per-CTA partial sums and the last-CTA counter.
// Set 0 is the default of every solve; sets 1 .. kRedSets - 1 serve concurrent set-up streams.
constexpr int kRedSets = 16;
struct RedSet {
    DevScalars* sc;
    double* partials;
    int64_t len;            // doubles available at `partials`
    unsigned int* counter;
};
RedSet red_set(pbm_grid* g, int rset);

// fine level: K(w) (u == nullptr) or S (u, d given; w = rho')
void launch_fine(pbm_grid* g, bool fp32, const void* w, const void* d, const void* u, const ApplyArgs& a,
                 cudaStream_t st);
// operator of level k (fine: K(rho) or S from the handle's data; coarse: the Galerkin matrices)
void level_apply(pbm_grid* g, int k, bool fp32, bool op_s, const ApplyArgs& a0, cudaStream_t st);
// coarse level k >= 1: explicit element matrices (+ border for S)
void launch_coarse(pbm_grid* g, int k, bool fp32, const ApplyArgs& a, cudaStream_t st);
// Jacobi diagonal of a level (S or K), written to L[k].diag64 / diag32 (n + 1, last = alpha)
void launch_diag(pbm_grid* g, int k, bool op_s, cudaStream_t st, int rset = 0, bool from32 = false);
// ------------------------------------------------------------------------------------------------
// batched launches: one launch covers several systems (grid handles); first[s] is the first CTA of
// system s (first[nsys] = total CTAs), sc[s] its scalar block; flags[1] == 0 marks a system whose
// solve is finished (its CTAs return at once)
// ------------------------------------------------------------------------------------------------
struct BatchMap {
    const int* first;
    DevScalars* const* sc;
    int nsys;
};
__device__ __forceinline__ int batch_system(const BatchMap& M, unsigned b) {
    int lo = 0, hi = M.nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (unsigned(M.first[mid]) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ bool batch_active(const BatchMap& M, int s) { return M.sc[s]->flags[1] != 0; }

// ---- launch arguments of the operator, transfer and coarse-solve kernels (single and batched) ----
template <class T>
struct ColArgs {
    int nx, ny, nz, support, L, nchunk;
    int64_t n, m, ncol;
    const T* x;        // gathered vector (n (+1))
    const T* w;        // element weights (fine)
    const T* d;        // Schur weights (fine S)
    const T* what;     // 21 x m transformed K_e u_e (fine S, table mode), row r = 7 c + q - 1
    const T* u;        // displacement (fine S, recompute mode)
    const T* A;        // coarse element matrices (300 x m, upper triangle, entry-major)
    KeHatT<T> K;
    T* QA;
    T* QB;
    double* apart;     // per-CTA partial sums of -t_e (fine S)
};

template <class T>
struct NodeArgs {
    int nx, ny, nz, support, L;
    int64_t n, ncol;
    const T* QA;
    const T* QB;
    const T* x;
    T* y;
    const T* b;
    const T* idiag;        // inverse Jacobi diagonal (JACOBI)
    const double* omega;   // device scalar (JACOBI)
    const T* bord;         // coarse alpha border (n) or nullptr
    const double* s_alpha; // coarse S_alpha,alpha (device scalar)
    int with_alpha;
    int mode;
    int dot_slot;
    const double* apart;   // pass-1 partials (fine S) or nullptr
    int napart;
    double* partials;      // 2 * gridDim.x
    DevScalars* sc;
    unsigned int* counter; // last-CTA counter
};

template <class T>
struct RestrictArgs {
    int nxf, nyf, nzf, support, with_alpha;
    const T* rf;
    T* bc;
    double scale;
    T* xfirst;
    const T* idiag;
    const double* om;
};

template <class T>
struct ProlongArgs {
    int nxf, nyf, nzf, support, with_alpha;
    const T* xc;
    T* xf;
};

template <class T>
struct CoarsestArgs {
    int N, n_vec;
    const double* Inv;
    const T* b;
    T* x;
};

// batched MINRES vector stages (krylov.cu): FIRST_JACOBI b = om f a (a input, f inverse diagonal);
// LANCZOS2 a = A z, b = v_prev, c = v_cur; UPDATE2 a = z_next, b = z, c = d_prev, d = d_prev2, e = x;
// ZERO b; COPY b = a
enum VecOp { VOP_FIRST_JACOBI = 0, VOP_LANCZOS2 = 1, VOP_UPDATE2 = 2, VOP_ZERO = 3, VOP_COPY = 4 };
enum ScalOp { SOP_INIT = 0, SOP_SCALARS = 1 };
template <class T>
struct VecArgs {
    int op;
    int64_t n;
    const T* a;
    T* b;
    T* c;
    T* d;
    T* e;
    const T* f;
    double* mr;
    const double* red;
    const double* om;
};
template <class T>
void launch_vec_b(const VecArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st);
void launch_scal_b(DevScalars* const* d_sc, int nsys, int op, cudaStream_t st);
template <class T>
RestrictArgs<T> make_restrict_args(pbm_grid* g, int k, const void* rf, void* bc, bool with_alpha, double scale,
                                   void* xfirst, int* blocks_out);
template <class T>
ProlongArgs<T> make_prolong_args(pbm_grid* g, int k, const void* xc, void* xf, bool with_alpha, int* blocks_out);
template <class T>
CoarsestArgs<T> make_coarsest_args(pbm_grid* g, const void* b, void* x, bool with_alpha, int* blocks_out);
template <class T>
void launch_restrict_b(const RestrictArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st);
template <class T>
void launch_prolong_b(const ProlongArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st);
template <class T>
void launch_coarsest_b(const CoarsestArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st);

// two-pass column kernels (colpass.cu). ColEnv names the scratch the passes use: the plane-quad
// buffers (cols_scratch_entries() entries of the vector type), the per-CTA partial sums and the
// device scalar block (last-CTA counter, reduction slots).
struct ColEnv {
    int L = 0;                 // chunk length of the fine column pass (0: the default rule)
    void* qa = nullptr;
    void* qb = nullptr;
    double* partials = nullptr;
    int64_t partials_len = 0;
    DevScalars* sc = nullptr;
    unsigned int* counter = nullptr;   // last-CTA counter (nullptr: &sc->counter[0])
};
int64_t cols_scratch_entries(const Geom& G);
ColEnv env_of(pbm_grid* g, int rset = 0);
// argument builders shared by the single and the batched launches (blocks_out: CTAs of the launch)
template <class T>
ColArgs<T> make_fine_args(const ColEnv& env, const Geom& G, const KeHat& kh, const T* w, const T* d, const T* what,
                          const T* u, const void* x, int* blocks_out);
template <class T>
ColArgs<T> make_coarse_args(const ColEnv& env, const Geom& G, const T* A, const void* x, int* blocks_out);
template <class T>
NodeArgs<T> make_node_args(const ColEnv& env, const Geom& G, const ApplyArgs& a, int L, const T* bord,
                           const double* s_alpha, const double* apart, int napart, int64_t off, int* blocks_out);
template <class T>
void launch_cols_fine_b(const ColArgs<T>* dA, const BatchMap& M, int mode, int total_blocks, cudaStream_t st);
template <class T>
void launch_cols_coarse_b(const ColArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st);
template <class T>
void launch_nodes_b(const NodeArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st);
template <class T>
void cols_fine_env(const ColEnv& env, const Geom& G, const KeHat& kh, const T* w, const T* d, const T* what,
                   const T* u, const ApplyArgs& a, cudaStream_t st);
// fine level: K(w) x (d == nullptr) or S (d given; W_e from `what` if given, else recomputed from u)
template <class T>
void cols_fine(pbm_grid* g, const T* w, const T* d, const T* what, const T* u, const ApplyArgs& a, cudaStream_t st);
template <class T>
void cols_coarse(pbm_grid* g, int k, const T* A, const T* bord, const ApplyArgs& a, cudaStream_t st,
                 bool per_element = false);
void launch_what_hat(pbm_grid* g, cudaStream_t st);
// single-pass FP32 fine operator (fused.cu): tile plan of candidate `cand` for a grid (of the K or the S
// operator), and the launch. The last plan is the tensor-core kernel (tc.cu).
struct FusedPlan {
    int TX, TY, DZ, gx, gy, gz;
    int var;   // kernel variant (threads per CTA, resident CTAs per SM; tensor cores)
};
FusedPlan fused_plan(const Geom& G, int cand, bool op_s = false);
int fused_num_plans();
int fused_tc_plan();
int fused_default_plan(const Geom& G);
int fused_blocks(const FusedPlan& p);
int fused_threads(const FusedPlan& p);
void fused_fine_f32(const FusedPlan& p, const RedSet& r, const Geom& G, const KeHat& kh, const TcMatrix& tm,
                    const float* w, const float* d, const float* u, const ApplyArgs& a, cudaStream_t st);
// tensor-core variant (tc.cu): operand matrices from K_e (host), plan, launch
void tc_build(const double* Ke, std::vector<float>& B, int& terms, float& scale);
FusedPlan tc_plan(const Geom& G, bool op_s);
void tc_fine_f32(const FusedPlan& p, const RedSet& r, const Geom& G, const TcMatrix& tm, const float* w,
                 const float* d, const float* u, const ApplyArgs& a, cudaStream_t st);
// lane-strip FP32 fine operator (strip.cu): plans cand = 0 .. strip_num_plans() - 1
int strip_num_plans();
int strip_threads(int cand);
FusedPlan strip_plan(const Geom& G, int cand);
void strip_fine_f32(int cand, const FusedPlan& p, const RedSet& r, const Geom& G, const KeHat& kh, const float* w,
                    const float* d, const float* u, const ApplyArgs& a, cudaStream_t st);
// single-pass FP32 coarse-level operator (stored Galerkin matrices; fused.cu)
int fused_coarse_num_plans();
FusedPlan fused_coarse_plan(const Geom& G, int cand);
void fused_coarse_f32(const FusedPlan& p, const RedSet& r, const Geom& G, const float* A, const float* bord,
                      const double* s_alpha, const ApplyArgs& a, cudaStream_t st);
void cols_cost(const Geom& G, int L, bool op_s, bool recompute_w, int mode, int esize, double& bytes, double& flops);
// chunk length the handle uses for the fine column pass of (precision, operator)
int fine_L(const pbm_grid* g, bool fp32, bool op_s);
// times the candidate chunk lengths of the fine column pass and keeps the fastest (grid creation)
void autotune_fine(pbm_grid* g);
// y = 1 / x and y = 1 / sqrt(x) (n entries)
void launch_inverse(const double* x, double* y, int64_t n, cudaStream_t st);
void launch_inverse_sqrt(const double* x, double* y, int64_t n, cudaStream_t st);
// per-element c_e = 1/2 u_e^T K_e u_e (masked u), FP64
void launch_elem_energy(pbm_grid* g, const double* u, const double* v, double* out, cudaStream_t st);
// profiling hooks around one fine-level operator launch (no-ops unless g->prof_on)
void prof_begin(pbm_grid* g, cudaStream_t st);
void prof_end(pbm_grid* g, cudaStream_t st, int op, double bytes, double flops);
void prof_fold(pbm_grid* g);

// ---- multigrid, mg.cu ----
// b_c = scale P^T r_f; if xfirst is given also xfirst = omega_{k+1} D_{k+1}^{-1} b_c (first Jacobi sweep)
void launch_restrict(pbm_grid* g, int k, bool fp32, const void* rf, void* bc, bool with_alpha, double scale,
                     cudaStream_t st, void* xfirst = nullptr);
void launch_prolong_add(pbm_grid* g, int k, bool fp32, const void* xc, void* xf, bool with_alpha, cudaStream_t st);
void launch_build_what(pbm_grid* g, cudaStream_t st, bool fp32);
void launch_build_level1(pbm_grid* g, bool op_s, cudaStream_t st, bool fp32);
void launch_build_coarser(pbm_grid* g, int k, cudaStream_t st, bool fp32);
void launch_coarse_to_f32(pbm_grid* g, int k, cudaStream_t st, bool matrices);
void launch_coarse_to_f64(pbm_grid* g, int k, cudaStream_t st);
// the FP64 Galerkin matrices and Jacobi diagonals of the coarse levels of a mixed grid (whose set-up
// builds them in FP32), built on first use by the calls that read them in FP64
void ensure_coarse64(pbm_grid* g, cudaStream_t st);
void build_coarsest(pbm_grid* g, bool op_s, cudaStream_t st);
void launch_coarsest_solve(pbm_grid* g, bool fp32, const void* b, void* x, bool with_alpha, cudaStream_t st);

// ---- vectors and reductions, krylov.cu ----
void vec_zero(void* p, size_t bytes, cudaStream_t st);
void launch_scale_diag_first(pbm_grid* g, int k, bool fp32, const void* b, void* x, bool with_alpha,
                             cudaStream_t st);                    // x = omega D^-1 b
void launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, cudaStream_t st);
void launch_dot(pbm_grid* g, bool fp32, const void* a, const void* b, int64_t n, int slot, cudaStream_t st);
double read_slot(pbm_grid* g, int slot, cudaStream_t st);

}  // namespace pbm
