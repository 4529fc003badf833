// Jacobi diagonals of the operators on a structured grid (the fine K(w) and S of eq. (S), and the
// stored coarse Galerkin operators), and the launch wrappers of the operator applications.
//
// The diagonals share one "marching" kernel. A CTA of 32 x BY threads covers 31 x (BY - 1) node
// columns of the grid and walks up a chunk of node planes in z. Thread (tx, ty) computes the
// diagonal contributions of the element whose upper corner (in x and y) is its own node column, one
// element layer per step:
//   * the element's contributions are split into its 4 bottom and 4 top corners: the top corners are
//     kept in registers and added to the next layer's bottom corners (same element column), so each
//     node plane is completed after two element layers;
//   * the 4 elements around a node column exchange their corner sums through shared memory and the
//     owning thread writes the node once: no atomics, and a fixed summation order (deterministic).
// Elements on CTA borders are computed twice (by the two CTAs that share them); the alpha entry of S
// (sum_i d_i) counts each element once and is finished by the last CTA from the per-CTA partial sums
// in a fixed order.
#include "pbm_internal.h"

namespace pbm {

enum Kind { K_FINE_DIAG_K = 2, K_FINE_DIAG_S = 3, K_COARSE_DIAG = 5 };

template <class T>
struct MarchParams {
    int nx, ny, nz, support, DZ;
    int64_t n, m;
    const T* w;        // element weights (fine level)
    const T* d;        // Schur weights (fine diagonal of S)
    const T* what_hat; // Khat H u_e of every fine element, [21][m] (fine diagonal of S)
    const T* A;        // coarse element matrices (upper triangle, entry-major)
    double s_alpha;    // S_alpha,alpha of a coarse level (the alpha entry of its diagonal)
    T* y;              // the diagonal, n (+ 1) entries
    int with_alpha;
    double Kdiag;      // K_e[i][i] of the fine element matrix
    double* partials;  // 2 * nblocks
    DevScalars* sc;
    unsigned int* counter;  // last-CTA counter
};

template <class T>
__device__ __forceinline__ T ldv(const T* p, int64_t i) { return __ldg(p + i); }

// deterministic block reduction of two values; result valid in thread 0
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
    const int lane = (threadIdx.x + blockDim.x * threadIdx.y) & 31;
    const int wid = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sh[2 * wid] = a;
        sh[2 * wid + 1] = b;
    }
    __syncthreads();
    if (wid == 0) {
        constexpr int NW = NT / 32;
        a = lane < NW ? sh[2 * lane] : 0.0;
        b = lane < NW ? sh[2 * lane + 1] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

template <class T, int BY, int KIND>
__global__ void __launch_bounds__(32 * BY) k_march(MarchParams<T> P) {
    constexpr int BX = 32;
    constexpr int NT = BX * BY;
    __shared__ T sacc[3][3][BY][BX];
    __shared__ double sred[2 * NT / 32];
    __shared__ bool s_last;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int X0 = blockIdx.x * (BX - 1), Y0 = blockIdx.y * (BY - 1);
    const int ex = X0 - 1 + tx, ey = Y0 - 1 + ty;
    const int Ix = X0 + tx, Iy = Y0 + ty;
    const bool owner = (tx < BX - 1) && (ty < BY - 1) && Ix <= nx && Iy <= ny;
    const bool ecol = ex >= 0 && ex < nx && ey >= 0 && ey < ny;
    const bool designated = ecol && tx >= 1 && ty >= 1;
    const int kz0 = blockIdx.z * P.DZ;
    const int kz1 = min(kz0 + P.DZ, nz + 1);
    const int64_t sxn = nx + 1, sxy = int64_t(nx + 1) * (ny + 1);

    T carry[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) carry[a][0] = carry[a][1] = carry[a][2] = T(0);
    double part_alpha = 0.0, part_zero = 0.0;

    for (int k = kz0 - 1; k < kz1; ++k) {
        __syncthreads();   // the owners have read the previous plane's corner sums
        T ye[3][8];
        const bool ev = ecol && k >= 0 && k < nz;
        if (ev) {
            const int64_t e = ex + int64_t(nx) * (ey + int64_t(ny) * k);
            if (KIND == K_FINE_DIAG_K) {
                const T we = ldv(P.w, e);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int a = 0; a < 8; ++a) ye[c][a] = we * T(P.Kdiag);
            } else if (KIND == K_FINE_DIAG_S) {
                const T we = ldv(P.w, e), de = ldv(P.d, e);
                // Khat H u_e from the table of the S pass (built from the masked u just before)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ye[c][0] = T(0);
#pragma unroll
                    for (int q = 1; q < 8; ++q) ye[c][q] = ldv(P.what_hat, int64_t(7 * c + q - 1) * P.m + e);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    wht_out(ye[c]);
#pragma unroll
                    for (int a = 0; a < 8; ++a) ye[c][a] = we * T(P.Kdiag) + de * ye[c][a] * ye[c][a];
                }
                if (designated && k >= kz0) part_alpha += double(de);
            } else {  // K_COARSE_DIAG
                const T* Ae = P.A + e;
                const int64_t m = P.m;
#pragma unroll
                for (int i = 0; i < 24; ++i) ye[i % 3][i / 3] = ldv(Ae, int64_t(tri_index(i, i)) * m);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 8; ++a) ye[c][a] = T(0);
        }

        // bottom corners complete node plane k (together with the layer below); top corners carry
        T acc[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[a][c] = carry[a][c] + ye[c][a];
                carry[a][c] = ye[c][a + 4];
            }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) sacc[a][c][ty][tx] = acc[a][c];
        __syncthreads();

        if (owner && k >= kz0 && k <= nz) {
            const int64_t nd = 3 * (Ix + sxn * Iy + sxy * k);
            const bool fixed = node_fixed(P.support, nx, ny, nz, Ix, Iy, k);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T yv = acc[3][c] + sacc[2][c][ty][tx + 1] + sacc[1][c][ty + 1][tx] + sacc[0][c][ty + 1][tx + 1];
                P.y[nd + c] = fixed ? T(1) : yv;   // identity rows of the supported dofs
            }
        }
    }

    // per-CTA partials, then the last CTA reduces them in order and writes the alpha entry
    block_sum2<NT>(part_alpha, part_zero, sred);
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tx == 0 && ty == 0) {
        P.partials[bid] = part_alpha;
        __threadfence();
        const unsigned t = atomicAdd(P.counter, 1u);
        s_last = (t == unsigned(nblk - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double sa = 0.0, sz = 0.0;
    const int tid = tx + BX * ty;
    sa = l2_strided_sum(P.partials, nblk, tid, NT);
    block_sum2<NT>(sa, sz, sred);
    if (tid == 0) {
        *P.counter = 0u;
        if (P.with_alpha) P.y[P.n] = T(KIND == K_COARSE_DIAG ? P.s_alpha : (KIND == K_FINE_DIAG_S ? sa : 1.0));
    }
}

// ------------------------------------------------------------------------------------------------
// launch helpers
// ------------------------------------------------------------------------------------------------
constexpr int BY_ = 8;

static dim3 march_grid(const Geom& g, int& DZ) {
    const int gx = (g.nx + 1 + 30) / 31;
    const int gy = (g.ny + 1 + BY_ - 2) / (BY_ - 1);
    const int planes = g.nz + 1;
    // aim for about 4 CTAs per SM, chunks of at least 4 planes
    const int want = num_sms() * 4;
    int chunks = (want + gx * gy - 1) / (gx * gy);
    chunks = std::max(1, std::min(chunks, (planes + 3) / 4));
    DZ = (planes + chunks - 1) / chunks;
    chunks = (planes + DZ - 1) / DZ;
    return dim3(gx, gy, chunks);
}

template <class T>
static void fill_khat(KeHatT<T>& out, const KeHat& K) {
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 8; ++q) out.dg[c][q] = T(K.dg[c][q]);
    for (int b = 0; b < 2; ++b) {
        out.lam4[b] = T(K.lam4[b]);
        out.mu4[b] = T(K.mu4[b]);
    }
}

template <class T>
static MarchParams<T> base_params(pbm_grid* g, int k, int rset = 0) {
    MarchParams<T> P{};
    const RedSet r = red_set(g, rset);
    const Geom& G = g->L[k].g;
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.support = G.support;
    P.n = G.n();
    P.m = G.m();
    P.partials = r.partials;
    P.sc = g->sc;
    P.counter = r.counter;
    P.Kdiag = g->Kdiag;
    return P;
}

template <class T, int KIND>
static void run(pbm_grid* g, int k, MarchParams<T>& P, cudaStream_t st, const char* what) {
    int DZ = 1;
    dim3 grid = march_grid(g->L[k].g, DZ);
    P.DZ = DZ;
    if (int(grid.x * grid.y * grid.z) > g->max_blocks) fail(PBM_EINVAL, "grid too large for the partials buffer");
    // (every reduction set holds at least 2 max_blocks partial sums)
    k_march<T, BY_, KIND><<<grid, dim3(32, BY_), 0, st>>>(P);
    PBM_LAUNCH(what);
}

// Fine-level operator applications: FP64 runs the two-pass column kernels (colpass.cu) with the
// W_e table, FP32 the single-pass kernel (fused.cu) that recomputes W_e from u. The marching kernel
// above builds the Jacobi diagonals.
void launch_fine(pbm_grid* g, bool fp32, const void* w, const void* d, const void* u, const ApplyArgs& a,
                 cudaStream_t st) {
    const bool s = u != nullptr;
    // profiling times the operator kernel of the grid's working precision (FP32 on mixed grids)
    const bool prof = g->prof_on && fp32 == (g->desc.precision == PBM_MIXED);
    if (prof) prof_begin(g, st);
    if (fp32)
        fused_fine_f32(fused_plan(g->L[0].g, g->fusedP[s ? 1 : 0], s), red_set(g, a.rset), g->L[0].g, g->kehat,
                       g->tc, (const float*)w, s ? (const float*)d : nullptr, s ? (const float*)u : nullptr, a, st);
    else
        cols_fine<double>(g, (const double*)w, s ? (const double*)d : nullptr, s ? g->what_hat : nullptr, nullptr, a,
                          st);
    if (prof) {
        double bytes = 0.0, flops = 0.0;
        cols_cost(g->L[0].g, fine_L(g, fp32, s), s, fp32, a.mode, fp32 ? 4 : 8, bytes, flops);
        prof_end(g, st, s ? PBM_OP_S : PBM_OP_K, bytes, flops);
    }
}

// Coarse levels. FP64 runs the two column passes (colpass.cu), whose finer split (eight threads per
// element) keeps the narrow FP64 pipe of every SM busy. FP32 runs, per level, whichever the grid's
// autotuner found faster: the single marching pass (fused.cu; one launch, tile halos read their
// element matrices twice) or the two passes with eight threads or one thread per element (no
// recomputation; the larger levels, where the matrices' traffic dominates).
void launch_coarse(pbm_grid* g, int k, bool fp32, const ApplyArgs& a, cudaStream_t st) {
    Level& L = g->L[k];
    const int plan = g->coarseP[a.with_alpha ? 1 : 0][k];
    if (fp32 && plan >= 0)
        fused_coarse_f32(fused_coarse_plan(L.g, plan), red_set(g, a.rset), L.g, L.A32, L.bord32, &g->sc->salpha, a,
                         st);
    else if (fp32)
        cols_coarse<float>(g, k, L.A32, L.bord32, a, st, plan == -2);
    else
        cols_coarse<double>(g, k, L.A64, L.bord64, a, st);
}

// FP64 Jacobi diagonal of coarse level k from its FP64 matrices into diag64
static void coarse_diag64(pbm_grid* g, int k, bool op_s, cudaStream_t st, int rset) {
    Level& L = g->L[k];
    auto P = base_params<double>(g, k, rset);
    P.with_alpha = 1;
    P.y = L.diag64;
    P.s_alpha = op_s ? g->s_alpha : 1.0;
    P.A = L.A64;
    run<double, K_COARSE_DIAG>(g, k, P, st, "coarse diag");
}

// from32: a coarse level of a mixed grid whose set-up built only the FP32 matrices (the diagonal is
// summed in FP32 and widened)
void launch_diag(pbm_grid* g, int k, bool op_s, cudaStream_t st, int rset, bool from32) {
    Level& L = g->L[k];
    if (k == 0) {
        auto P = base_params<double>(g, k, rset);
        P.with_alpha = 1;
        P.y = L.diag64;
        P.s_alpha = g->s_alpha;
        P.w = op_s ? g->w64 : g->rho;
        if (op_s) {
            P.d = g->d64;
            P.what_hat = g->what_hat;   // filled by launch_what_hat before the diagonal
            run<double, K_FINE_DIAG_S>(g, 0, P, st, "fine diag S");
        } else {
            run<double, K_FINE_DIAG_K>(g, 0, P, st, "fine diag K");
        }
    } else if (from32) {
        auto P = base_params<float>(g, k, rset);
        P.with_alpha = 1;
        P.y = L.t32;
        P.s_alpha = op_s ? g->s_alpha : 1.0;
        P.A = L.A32;
        run<float, K_COARSE_DIAG>(g, k, P, st, "coarse diag");
        launch_cast(L.t32, true, L.diag64, false, L.g.n() + 1, st);
    } else {
        coarse_diag64(g, k, op_s, st, rset);
    }
    launch_inverse(L.diag64, L.idiag64, L.g.n() + 1, st);
    if (L.idiag32) launch_cast(L.idiag64, false, L.idiag32, true, L.g.n() + 1, st);
}

void ensure_coarse64(pbm_grid* g, cudaStream_t st) {
    if (g->desc.precision != PBM_MIXED || g->coarse64_ready || g->levels < 2 || g->op_ready == 0) return;
    const bool op_s = g->op_ready == 2;
    if (op_s) launch_build_what(g, st, false);
    launch_build_level1(g, op_s, st, false);
    for (int k = 1; k + 1 < g->levels; ++k) launch_build_coarser(g, k, st, false);
    // the FP64 diagonals only: the FP32 smoother keeps the weights and inverse diagonals of its set-up
    for (int k = 1; k < g->levels; ++k) coarse_diag64(g, k, op_s, st, 0);
    g->coarse64_ready = true;
}

// ------------------------------------------------------------------------------------------------
// per-element bilinear forms u_e^T K_e v_e with supported dofs masked (fine level)
// ------------------------------------------------------------------------------------------------
__global__ void k_elem_energy(int nx, int ny, int nz, int support, const double* __restrict__ u,
                              const double* __restrict__ v, double* __restrict__ out, KeHatT<double> K) {
    const int64_t m = int64_t(nx) * ny * nz;
    const int64_t sxn = nx + 1, sxy = int64_t(nx + 1) * (ny + 1);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(e % nx);
        const int j = int((e / nx) % ny);
        const int k = int(e / (int64_t(nx) * ny));
        double U[3][8], X[3][8], W[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + ((a >> 2) & 1);
            const bool fx = node_fixed(support, nx, ny, nz, ii, jj, kk);
            const int64_t nd = 3 * (ii + sxn * jj + sxy * kk);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                U[c][a] = fx ? 0.0 : u[nd + c];
                X[c][a] = fx ? 0.0 : v[nd + c];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            wht_fwd(U[c]);
            wht_fwd(X[c]);
        }
        khat_apply(K, U, W);
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 1; q < 8; ++q) s += W[c][q] * X[c][q];
        out[e] = s;
    }
}

void launch_elem_energy(pbm_grid* g, const double* u, const double* v, double* out, cudaStream_t st) {
    const Geom& G = g->L[0].g;
    KeHatT<double> K;
    fill_khat(K, g->kehat);
    const int64_t m = G.m();
    int blocks = int(std::min<int64_t>((m + 255) / 256, num_sms() * 16));
    k_elem_energy<<<blocks, 256, 0, st>>>(G.nx, G.ny, G.nz, G.support, u, v ? v : u, out, K);
    PBM_LAUNCH("elem energy");
}

}  // namespace pbm
