// Two-pass operator application: element columns, then nodes.
//
// Pass 1 gives every thread one element column (i, j) and a chunk of L element layers of it (the
// coarse levels use L = 1 and split each element's 24 rows over eight threads, or, on FP32 levels
// where the autotuner finds it faster, give each thread one element). For each layer it
// forms the element's contribution to the 8 corner nodes and writes, per node plane, the 4 corner
// values of the column ("plane quads") to scratch:
//   QA[k]  plane k as bottom face of layer k (plus, inside a chunk, the top face of layer k - 1),
//   QB[c]  the top face of the last layer of chunk c (plane min((c + 1) L, nz)).
// Pass 2 gives every thread one node, sums the quads of the (up to) four columns around it in a
// fixed order and applies the epilogue (plain apply, residual b - A x, damped-Jacobi sweep), the
// dot products of the Krylov solvers and, for S, the alpha row. No element is computed twice, no
// atomics are used and the summation order is fixed, so results are bit-reproducible.
//
// On the fine level the element matrix is applied in the factored form K_e = H^T Khat H (see
// pbm_internal.h). The forward transform is split: the xy part of each node plane's quad is
// computed once and shared by the two element layers that touch the plane, the z part is per
// element; the inverse transform runs the z part per element, adds the top face of the layer below
// (same thread), and the xy part once per plane. For S the transformed vector W_e = Khat H u_e is
// read from a table built at set-up (pbm_set_state), so the rank-one term costs a dot product and
// an axpy of 21 coefficients:  Y_e = rho'_e Khat X_e + t_e W_e,  t_e = d_e (W_e . X_e - x_alpha).
//
// This is the FP64 path: GB300 issues about two FP64 operations per clock per SM, so the FP64
// operator is bound by the FP64 pipe, not by HBM; the split removes the halo elements that a
// tiled single pass recomputes and lets every SM take an equal share of the columns.
#include "pbm_internal.h"

namespace pbm {

constexpr int CB = 128;   // threads per pass-1 CTA
constexpr int NB2 = 256;  // threads per pass-2 CTA

// forward xy transform of the masked node quad (i .. i+1, j .. j+1) of plane k of vector v
template <class T>
__device__ __forceinline__ void load_quad(const ColArgs<T>& P, const T* __restrict__ vec, int i, int j, int k,
                                          T (&Q)[3][4]) {
    const int64_t sxn = P.nx + 1, sxy = int64_t(P.nx + 1) * (P.ny + 1);
    T v[3][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int ii = i + (a & 1), jj = j + (a >> 1);
        const bool fx = node_fixed(P.support, P.nx, P.ny, P.nz, ii, jj, k);
        const int64_t nd = 3 * (ii + sxn * jj + sxy * k);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][a] = fx ? T(0) : __ldg(vec + nd + c);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T s0 = v[c][0] + v[c][1], d0 = v[c][1] - v[c][0];
        const T s1 = v[c][2] + v[c][3], d1 = v[c][3] - v[c][2];
        Q[c][0] = s0 + s1;
        Q[c][1] = d0 + d1;
        Q[c][2] = s1 - s0;
        Q[c][3] = d1 - d0;
    }
}

template <class T>
__device__ __forceinline__ void load_quad(const ColArgs<T>& P, int i, int j, int k, T (&Q)[3][4]) {
    load_quad(P, P.x, i, j, k, Q);
}

// inverse xy transform of a transformed plane quad, stored as nodal corner values
template <class T>
__device__ __forceinline__ void store_quad(T* Q, int64_t slot, int64_t ncol, int64_t col, const T (&V)[3][4]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T a0 = V[c][0] - V[c][1], a1 = V[c][0] + V[c][1];
        const T a2 = V[c][2] - V[c][3], a3 = V[c][2] + V[c][3];
        T* q = Q + (slot * 12 + c) * ncol + col;
        q[0] = a0 - a2;           // corner 0 (i,   j)
        q[3 * ncol] = a1 - a3;    // corner 1 (i+1, j)
        q[6 * ncol] = a0 + a2;    // corner 2 (i,   j+1)
        q[9 * ncol] = a1 + a3;    // corner 3 (i+1, j+1)
    }
}

template <int NT>
__device__ __forceinline__ double cta_sum1(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += sh[w];
    return s;
}

// ------------------------------------------------------------------------------------------------
// pass 1, fine level: K(w) x (S = false) or the S operator (S = true)
// ------------------------------------------------------------------------------------------------
// MODE 0: K(w) x. MODE 1: S with W_e read from the table (FP64). MODE 2: S with W_e recomputed
// from the plane quads of u (FP32: the recomputation costs ALU the FP32 pipe has to spare, the
// table would cost 21 values per element of HBM traffic).
template <class T, int MODE>
__device__ __forceinline__ void cols_fine_body(const ColArgs<T>& P, unsigned blk) {
    constexpr bool S = MODE != 0;
    __shared__ double sh[CB / 32];
    const int64_t tid = blk * int64_t(CB) + threadIdx.x;
    T apartT = T(0);
    if (tid < P.ncol * P.nchunk) {
        const unsigned ncol = unsigned(P.ncol), nxu = unsigned(P.nx);
        const unsigned chunk_u = unsigned(tid) / ncol;
        const unsigned colu = unsigned(tid) - chunk_u * ncol;
        const int64_t col = colu;
        const int chunk = int(chunk_u);
        const int j = int(colu / nxu), i = int(colu - unsigned(j) * nxu);
        const int k0 = chunk * P.L, k1 = min(k0 + P.L, P.nz);
        const T xa = S ? P.x[P.n] : T(0);
        T Qlo[3][4], Qhi[3][4], carry[3][4];
        T Ulo[3][4], Uhi[3][4];
        load_quad(P, i, j, k0, Qlo);
        if (MODE == 2) load_quad(P, P.u, i, j, k0, Ulo);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 4; ++q) carry[c][q] = T(0);
        for (int k = k0; k < k1; ++k) {
            load_quad(P, i, j, k + 1, Qhi);
            if (MODE == 2) load_quad(P, P.u, i, j, k + 1, Uhi);
            const int64_t e = col + P.ncol * k;
            T X[3][8], Y[3][8];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    X[c][q] = Qlo[c][q] + Qhi[c][q];
                    X[c][q + 4] = Qhi[c][q] - Qlo[c][q];
                }
            khat_apply(P.K, X, Y);
            const T we = __ldg(P.w + e);
            if (S) {
                T Wt[3][8];
                if (MODE == 2) {
                    T U[3][8];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            U[c][q] = Ulo[c][q] + Uhi[c][q];
                            U[c][q + 4] = Uhi[c][q] - Ulo[c][q];
                            Ulo[c][q] = Uhi[c][q];
                        }
                    khat_apply(P.K, U, Wt);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        Wt[c][0] = T(0);
#pragma unroll
                        for (int q = 1; q < 8; ++q) Wt[c][q] = __ldg(P.what + int64_t(7 * c + q - 1) * P.m + e);
                    }
                }
                T dot = T(0);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int q = 1; q < 8; ++q) dot += Wt[c][q] * X[c][q];
                const T t = __ldg(P.d + e) * (dot - xa);
                apartT -= t;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int q = 1; q < 8; ++q) Y[c][q] = we * Y[c][q] + t * Wt[c][q];
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int q = 1; q < 8; ++q) Y[c][q] *= we;
            }
            // z part of the inverse transform: bottom face (plane k) and top face (plane k + 1)
            T Bq[3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    Bq[c][q] = carry[c][q] + (Y[c][q] - Y[c][q + 4]);
                    carry[c][q] = Y[c][q] + Y[c][q + 4];
                    Qlo[c][q] = Qhi[c][q];
                }
            store_quad(P.QA, k, P.ncol, col, Bq);
        }
        store_quad(P.QB, chunk, P.ncol, col, carry);
    }
    if (S) {
        const double s = cta_sum1<CB>(double(apartT), sh);
        if (threadIdx.x == 0) P.apart[blk] = s;
    }
}

template <class T, int MODE>
__global__ void __launch_bounds__(CB) k_cols_fine(ColArgs<T> P) {
    pdl_wait();
    cols_fine_body<T, MODE>(P, blockIdx.x);
}

template <class T, int MODE>
__global__ void __launch_bounds__(CB) k_cols_fine_b(const ColArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    cols_fine_body<T, MODE>(A[s], blockIdx.x - M.first[s]);
}

// ------------------------------------------------------------------------------------------------
// pass 1, coarse levels: explicit element matrices. Thread (e, a) forms the 3 rows of local node a
// of element e (72 FMAs): FP64 work per thread stays short, so the small coarse levels are not
// limited by one thread's chain of dependent FP64 instructions. Threads of one warp share a, so
// the matrix reads (entry-major) are coalesced over consecutive elements.
// ------------------------------------------------------------------------------------------------
template <class T, int A>
__device__ __forceinline__ void coarse_node_rows(const T* __restrict__ Ae, int64_t m, const T (&xe)[24], T (&y)[3]) {
    // all 72 entries are loaded before the sums (one round of loads: on the small coarse levels the pass is bound
    // by load latency), then summed in the fixed order
    T av[3][24];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int r = 3 * A + c;
#pragma unroll
        for (int s = 0; s < 24; ++s) {
            const int t = r <= s ? tri_index(r, s) : tri_index(s, r);
            av[c][s] = __ldg(Ae + int64_t(t) * m);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < 24; ++s) acc += av[c][s] * xe[s];
        y[c] = acc;
    }
}

template <class T>
__device__ __forceinline__ void cols_coarse_body(const ColArgs<T>& P, unsigned blk) {
    const unsigned tid = blk * CB + threadIdx.x;
    const unsigned mu = unsigned(P.m), ncol = unsigned(P.ncol), nxu = unsigned(P.nx);
    if (tid >= 8 * mu) return;
    const int a = int(tid / mu);
    const unsigned eu = tid - unsigned(a) * mu;
    const unsigned ku = eu / ncol, colu = eu - ku * ncol;
    const int64_t e = eu, col = colu;
    const int k = int(ku);
    const int j = int(colu / nxu), i = int(colu - unsigned(j) * nxu);
    const int64_t sxn = P.nx + 1, sxy = int64_t(P.nx + 1) * (P.ny + 1);
    T xe[24];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int ii = i + (b & 1), jj = j + ((b >> 1) & 1), kk = k + (b >> 2);
        const bool fx = node_fixed(P.support, P.nx, P.ny, P.nz, ii, jj, kk);
        const int64_t nd = 3 * (ii + sxn * jj + sxy * kk);
#pragma unroll
        for (int c = 0; c < 3; ++c) xe[3 * b + c] = fx ? T(0) : __ldg(P.x + nd + c);
    }
    T y[3];
    switch (a) {
        case 0: coarse_node_rows<T, 0>(P.A + e, P.m, xe, y); break;
        case 1: coarse_node_rows<T, 1>(P.A + e, P.m, xe, y); break;
        case 2: coarse_node_rows<T, 2>(P.A + e, P.m, xe, y); break;
        case 3: coarse_node_rows<T, 3>(P.A + e, P.m, xe, y); break;
        case 4: coarse_node_rows<T, 4>(P.A + e, P.m, xe, y); break;
        case 5: coarse_node_rows<T, 5>(P.A + e, P.m, xe, y); break;
        case 6: coarse_node_rows<T, 6>(P.A + e, P.m, xe, y); break;
        default: coarse_node_rows<T, 7>(P.A + e, P.m, xe, y); break;
    }
    // bottom nodes (a < 4) go to QA[k], top nodes to QB[k]; corner a & 3
    T* Q = (a < 4 ? P.QA : P.QB) + (int64_t(k) * 12 + 3 * (a & 3)) * P.ncol + col;
#pragma unroll
    for (int c = 0; c < 3; ++c) Q[c * P.ncol] = y[c];
}

template <class T>
__global__ void __launch_bounds__(CB, 4) k_cols_coarse(ColArgs<T> P) {
    pdl_wait();
    pdl_launch_if_small();
    cols_coarse_body<T>(P, blockIdx.x);
}

// The same pass with one thread per element (FP32 levels whose matrices dominate the traffic):
// each stored entry (r, s), r <= s, is loaded once and used twice (y_r += a x_s, y_s += a x_r), so
// the SMs load 300 values per element instead of the 576 the row-wise split reads (every entry
// off the diagonal by two threads). Lanes are consecutive elements, so every load of an entry is
// one coalesced row of the entry-major array; the eight corner rows go to the same plane-quad
// scratch as the split pass, and the node pass is shared.
template <class T>
__global__ void __launch_bounds__(CB, 4) k_cols_coarse_e(ColArgs<T> P) {
    pdl_wait();
    pdl_launch_if_small();
    const unsigned mu = unsigned(P.m), ncol = unsigned(P.ncol), nxu = unsigned(P.nx);
    const unsigned eu = blockIdx.x * CB + threadIdx.x;
    if (eu >= mu) return;
    const unsigned ku = eu / ncol, colu = eu - ku * ncol;
    const int k = int(ku);
    const int j = int(colu / nxu), i = int(colu - unsigned(j) * nxu);
    const int64_t sxn = P.nx + 1, sxy = int64_t(P.nx + 1) * (P.ny + 1);
    T xe[24], y[24];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int ii = i + (b & 1), jj = j + ((b >> 1) & 1), kk = k + (b >> 2);
        const bool fx = node_fixed(P.support, P.nx, P.ny, P.nz, ii, jj, kk);
        const int64_t nd = 3 * (ii + sxn * jj + sxy * kk);
#pragma unroll
        for (int c = 0; c < 3; ++c) xe[3 * b + c] = fx ? T(0) : __ldg(P.x + nd + c);
    }
#pragma unroll
    for (int r = 0; r < 24; ++r) y[r] = T(0);
    const T* Ae = P.A + eu;
    // row r of the upper triangle (its entries are consecutive in the entry order) is loaded two rows ahead of
    // its use, so that about two rows of loads per thread are in flight while a row is multiplied (the matrices
    // are read once, from DRAM: the pass is bound by how many loads the SM keeps in flight)
    T a[3][24];
    auto load_row = [&](int r, T (&dst)[24]) {
#pragma unroll
        for (int s = r; s < 24; ++s) dst[s] = __ldg(Ae + int64_t(tri_index(r, s)) * mu);
    };
    load_row(0, a[0]);
    load_row(1, a[1]);
#pragma unroll
    for (int r = 0; r < 24; ++r) {
        if (r + 2 < 24) load_row(r + 2, a[(r + 2) % 3]);
        const T (&ar)[24] = a[r % 3];
        y[r] += ar[r] * xe[r];
#pragma unroll
        for (int s = r + 1; s < 24; ++s) {
            y[r] += ar[s] * xe[s];
            y[s] += ar[s] * xe[r];
        }
    }
    const int64_t col = colu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        T* Q = (b < 4 ? P.QA : P.QB) + (int64_t(k) * 12 + 3 * (b & 3)) * P.ncol + col;
#pragma unroll
        for (int c = 0; c < 3; ++c) Q[c * P.ncol] = y[3 * b + c];
    }
}

template <class T>
__global__ void __launch_bounds__(CB, 4) k_cols_coarse_b(const ColArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    cols_coarse_body<T>(A[s], blockIdx.x - M.first[s]);
}

// ------------------------------------------------------------------------------------------------
// pass 2: node sums, epilogue, dots, alpha row
// ------------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void nodes_body(const NodeArgs<T>& P, unsigned blk, unsigned nblk) {
    __shared__ double sh[NB2 / 32];
    __shared__ bool s_last;
    const int nx = P.nx, ny = P.ny, nz = P.nz, L = P.L;
    // node counts stay below 2^31 (checked at grid creation): 32-bit index arithmetic
    const unsigned nn = unsigned(P.n / 3);
    const unsigned sx = unsigned(nx + 1), sy = unsigned(ny + 1);
    const T xa = P.with_alpha ? P.x[P.n] : T(0);
    // epilogue weights, converted once and only in their mode
    T omT = T(0), c0T = T(0), c1T = T(0), c2T = T(0);
    bool c1nz = false;
    if (P.mode == EPI_JACOBI) omT = T(*P.omega);
    if (P.mode == EPI_CHEB) {
        c0T = T(P.omega[0]);
        c1T = T(P.omega[1]);
        c2T = T(P.omega[2]);
        c1nz = c1T != T(0);
    }
    // per-thread partial sums in the vector type (no FP64 work per entry in the FP32 kernels), the
    // dot product only when the launch asks for it
    const bool want_dot = P.dot_slot >= 0;
    T pdT = T(0), paT = T(0);
    for (unsigned nd = blk * NB2 + threadIdx.x; nd < nn; nd += nblk * NB2) {
        const unsigned r = nd / sx;
        const int I = int(nd - r * sx), J = int(r % sy), K = int(r / sy);
        const bool hasA = K < nz;
        const bool hasB = K > 0 && (K % L == 0 || K == nz);
        const int64_t oa = int64_t(K) * 12 * P.ncol, ob = int64_t(K > 0 ? (K - 1) / L : 0) * 12 * P.ncol;
        const int64_t d0 = 3 * int64_t(nd);
        // every load of the node first (the quads of the four columns around it, its x and the
        // epilogue's operands), then the sums in a fixed order
        T qa[4][3], qb[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int dj = 1 - (q >> 1), di = 1 - (q & 1);
            const int ii = I - di, jj = J - dj;
            const bool in = ii >= 0 && ii < nx && jj >= 0 && jj < ny;
            const int64_t col = in ? ii + int64_t(nx) * jj : 0;
            const int a = di + 2 * dj;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t r = int64_t(3 * a + c) * P.ncol + col;
                qa[q][c] = (in && hasA) ? __ldg(P.QA + oa + r) : T(0);
                qb[q][c] = (in && hasB) ? __ldg(P.QB + ob + r) : T(0);
            }
        }
        T xo[3], bv[3] = {T(0), T(0), T(0)}, dv[3] = {T(0), T(0), T(0)}, yp[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xo[c] = P.x[d0 + c];
            if (P.mode != EPI_APPLY) bv[c] = __ldg(P.b + d0 + c);
            if (P.mode >= EPI_JACOBI) dv[c] = __ldg(P.idiag + d0 + c);
            if (c1nz) yp[c] = P.y[d0 + c];
        }
        T s[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                s[c] += qa[q][c];
                s[c] += qb[q][c];
            }
        const bool fixed = node_fixed(P.support, nx, ny, nz, I, J, K);
        if (P.bord) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T bc = P.bord[d0 + c];
                s[c] += bc * xa;
                paT += bc * xo[c];
            }
        }
        if (fixed) {
            s[0] = xo[0];
            s[1] = xo[1];
            s[2] = xo[2];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T o;
            if (P.mode == EPI_APPLY) {
                o = s[c];
                if (want_dot) pdT += o * xo[c];
            } else if (P.mode == EPI_RESID) {
                o = bv[c] - s[c];
                if (want_dot) pdT += o * o;
            } else if (P.mode == EPI_JACOBI) {
                o = xo[c] + omT * ((bv[c] - s[c]) * dv[c]);
                if (want_dot) pdT += o * bv[c];
            } else if (P.mode == EPI_CHEB) {
                o = c0T * xo[c] + c2T * ((bv[c] - s[c]) * dv[c]);
                if (c1nz) o -= c1T * yp[c];
                if (want_dot) pdT += o * bv[c];
            } else {
                o = (3 * node_colour(I, J, K) + c == P.mode - EPI_GS0) ? xo[c] + (bv[c] - s[c]) * dv[c] : xo[c];
                if (want_dot) pdT += o * bv[c];
            }
            P.y[d0 + c] = o;
        }
    }
    const double pd = double(pdT), pa = double(paT);
    // per-CTA partials, then the last CTA finishes the alpha entry and the dot in a fixed order
    // (skipped when the launch needs neither: smoothing sweeps and residuals of K inside the V-cycle)
    if (P.dot_slot < 0 && !P.with_alpha) return;
    const double bd = cta_sum1<NB2>(pd, sh);
    __syncthreads();
    const double ba = cta_sum1<NB2>(pa, sh);
    if (threadIdx.x == 0) {
        P.partials[blk] = bd;
        P.partials[nblk + blk] = ba;
        __threadfence();
        s_last = atomicAdd(P.counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // every thread of the last CTA sums a fixed strided subset; the CTA sum has a fixed tree order
    double td = 0.0, ta = 0.0;
    td = l2_strided_sum(P.partials, int(nblk), threadIdx.x, NB2);
    ta = l2_strided_sum(P.partials + nblk, int(nblk), threadIdx.x, NB2);
    if (P.apart) {
        // continues this thread's alpha share in the same order
        for (int q0 = threadIdx.x; q0 < P.napart; q0 += 8 * NB2) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = q0 + u * NB2 < P.napart ? __ldcg(P.apart + q0 + u * NB2) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (q0 + u * NB2 < P.napart) ta += v[u];
        }
    }
    __syncthreads();
    double sd = cta_sum1<NB2>(td, sh);
    __syncthreads();
    double sa = cta_sum1<NB2>(ta, sh);
    if (threadIdx.x != 0) return;
    *P.counter = 0u;
    if (P.with_alpha) {
        const int64_t n = P.n;
        const double ya = sa + (P.bord ? *P.s_alpha * double(xa) : 0.0);
        double o;
        if (P.mode == EPI_APPLY) {
            o = ya;
            sd += o * double(xa);
        } else if (P.mode == EPI_RESID) {
            o = double(P.b[n]) - ya;
            sd += o * o;
        } else if (P.mode == EPI_JACOBI) {
            const double bb = double(P.b[n]);
            o = double(xa) + *P.omega * ((bb - ya) * double(P.idiag[n]));
            sd += o * bb;
        } else if (P.mode == EPI_CHEB) {
            const double bb = double(P.b[n]);
            o = P.omega[0] * double(xa) + P.omega[2] * ((bb - ya) * double(P.idiag[n]));
            if (P.omega[1] != 0.0) o -= P.omega[1] * double(P.y[n]);
            sd += o * bb;
        } else {
            const double bb = double(P.b[n]);
            o = P.mode == EPI_GS0 + kGsColours ? double(xa) + (bb - ya) * double(P.idiag[n]) : double(xa);
            sd += o * bb;
        }
        P.y[n] = T(o);
    }
    if (P.dot_slot >= 0) P.sc->red[P.dot_slot] = sd;
}

template <class T>
__global__ void __launch_bounds__(NB2) k_nodes(NodeArgs<T> P) {
    pdl_wait();
    pdl_launch_if_small();
    nodes_body<T>(P, blockIdx.x, gridDim.x);
}

template <class T>
__global__ void __launch_bounds__(NB2) k_nodes_b(const NodeArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    nodes_body<T>(A[s], blockIdx.x - M.first[s], M.first[s + 1] - M.first[s]);
}

// ------------------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------------------
// chunk length of the fine pass: the longest of 8, 4, 2, 1 layers that still gives every SM
// sub-partition (4 per SM) at least two warps of columns
static int fine_chunk(const Geom& G) {
    const int64_t ncol = int64_t(G.nx) * G.ny;
    const int64_t want = int64_t(num_sms()) * 4 * 32 * 2;
    for (int L = 8; L > 1; L >>= 1)
        if (ncol * ((G.nz + L - 1) / L) >= want) return L;
    return 1;
}

template <class T>
NodeArgs<T> make_node_args(const ColEnv& env, const Geom& G, const ApplyArgs& a, int L, const T* bord,
                           const double* s_alpha, const double* apart, int napart, int64_t off, int* blocks_out) {
    NodeArgs<T> N{};
    N.nx = G.nx;
    N.ny = G.ny;
    N.nz = G.nz;
    N.support = G.support;
    N.L = L;
    N.n = G.n();
    N.ncol = int64_t(G.nx) * G.ny;
    N.QA = (const T*)env.qa;
    N.QB = (const T*)env.qb;
    N.x = (const T*)a.x;
    N.y = (T*)a.y;
    N.b = (const T*)a.b;
    N.idiag = (const T*)a.diag;
    N.omega = a.omega;
    N.bord = a.with_alpha ? bord : nullptr;
    N.s_alpha = s_alpha;
    N.with_alpha = a.with_alpha ? 1 : 0;
    N.mode = a.mode;
    N.dot_slot = a.dot_slot;
    N.apart = apart;
    N.napart = napart;
    N.partials = env.partials + off;
    N.sc = env.sc;
    N.counter = env.counter ? env.counter : &env.sc->counter[0];
    const int64_t nn = G.nnode();
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((nn + NB2 - 1) / NB2, int64_t(num_sms()) * kNodeBlocksPerSm)));
    if (off + 2 * blocks > env.partials_len) fail(PBM_EINVAL, "grid too large for the partials buffer");
    *blocks_out = blocks;
    return N;
}

template <class T>
static void node_pass(const ColEnv& env, const Geom& G, const ApplyArgs& a, int L, const T* bord,
                      const double* s_alpha, const double* apart, int napart, int64_t off, cudaStream_t st) {
    int blocks = 0;
    NodeArgs<T> N = make_node_args<T>(env, G, a, L, bord, s_alpha, apart, napart, off, &blocks);
    launch_pdl(k_nodes<T>, dim3(blocks), dim3(NB2), 0, st, N);
    PBM_LAUNCH("node pass");
}

template <class T>
static void fill_khat_t(KeHatT<T>& out, const KeHat& K) {
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 8; ++q) out.dg[c][q] = T(K.dg[c][q]);
    for (int b = 0; b < 2; ++b) {
        out.lam4[b] = T(K.lam4[b]);
        out.mu4[b] = T(K.mu4[b]);
    }
}

// Algorithmic cost of one fine-level operator application by the column passes (profiling
// statistics). Bytes: every input vector and element array read once, the output written once
// (the quad scratch is not algorithmic). Operations (add, mul, FMA each counted once) per element:
// xy transforms of the plane quads 24 (L + 1) / L in and out, z transforms 24 in and out, Khat 45,
// scaling by the weight 21, carry 12 (L - 1) / L; S adds the dot W.X 21, t_e 2 and the axpy t W 21,
// and, when W_e is recomputed from u, the transforms and Khat of u.
// Per node: 12 quad sums plus the epilogue (apply 3, residual 6, Jacobi 12).
void cols_cost(const Geom& G, int Lc, bool op_s, bool recompute_w, int mode, int esize, double& bytes, double& flops) {
    const double n = double(G.n()), m = double(G.m()), nn = double(G.nnode());
    double vec = 2.0 * n + (op_s ? n : 0.0), elem = m * (op_s ? 2.0 : 1.0);
    if (mode == EPI_RESID) vec += n;
    if (mode == EPI_JACOBI) vec += 2.0 * n;
    if (mode == EPI_CHEB) vec += 3.0 * n;   // b, the inverse diagonal and the previous iterate
    if (mode >= EPI_GS0) vec += 2.0 * n;    // a Gauss-Seidel colour step: b and the inverse diagonal
    bytes = double(esize) * (vec + elem);
    const double L = double(Lc > 0 ? Lc : fine_chunk(G));
    double per_elem = 2.0 * 24.0 * (L + 1.0) / L + 48.0 + 45.0 + 21.0 + 12.0 * (L - 1.0) / L;
    if (op_s) per_elem += 44.0;
    if (op_s && recompute_w) per_elem += 24.0 * (L + 1.0) / L + 24.0 + 45.0;   // quads, z part and Khat of u
    const double per_node =
        12.0 + (mode == EPI_CHEB ? 18.0 : (mode == EPI_JACOBI ? 12.0 : (mode == EPI_RESID ? 6.0 : 3.0)));
    flops = m * per_elem + nn * per_node;
}

template <class T>
ColArgs<T> make_fine_args(const ColEnv& env, const Geom& G, const KeHat& kh, const T* w, const T* d, const T* what,
                          const T* u, const void* x, int* blocks_out) {
    ColArgs<T> P{};
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.support = G.support;
    P.L = env.L > 0 ? env.L : fine_chunk(G);
    P.nchunk = (G.nz + P.L - 1) / P.L;
    P.n = G.n();
    P.m = G.m();
    P.ncol = int64_t(G.nx) * G.ny;
    P.x = (const T*)x;
    P.w = w;
    P.d = d;
    P.what = what;
    P.u = u;
    fill_khat_t(P.K, kh);
    P.QA = (T*)env.qa;
    P.QB = (T*)env.qb;
    P.apart = env.partials;
    const int64_t threads = P.ncol * P.nchunk;
    const int blocks = int((threads + CB - 1) / CB);
    if (d && blocks > env.partials_len / 2) fail(PBM_EINVAL, "grid too large for the partials buffer");
    *blocks_out = blocks;
    return P;
}

template <class T>
void cols_fine_env(const ColEnv& env, const Geom& G, const KeHat& kh, const T* w, const T* d, const T* what,
                   const T* u, const ApplyArgs& a, cudaStream_t st) {
    int blocks = 0;
    const ColArgs<T> P = make_fine_args<T>(env, G, kh, w, d, what, u, a.x, &blocks);
    const bool s = d != nullptr;
    if (s && what) launch_pdl(k_cols_fine<T, 1>, dim3(blocks), dim3(CB), 0, st, P);
    else if (s) launch_pdl(k_cols_fine<T, 2>, dim3(blocks), dim3(CB), 0, st, P);
    else launch_pdl(k_cols_fine<T, 0>, dim3(blocks), dim3(CB), 0, st, P);
    PBM_LAUNCH("fine column pass");
    node_pass<T>(env, G, a, P.L, (const T*)nullptr, nullptr, s ? env.partials : nullptr, s ? blocks : 0,
                 s ? blocks : 0, st);
}

int64_t cols_scratch_entries(const Geom& G) {
    const int64_t ncol = int64_t(G.nx) * G.ny;
    const int L = fine_chunk(G);
    return 12 * ncol * (G.nz + 1) + 12 * ncol * ((G.nz + L - 1) / L);
}

ColEnv env_of(pbm_grid* g, int rset) {
    const RedSet r = red_set(g, rset);
    ColEnv e;
    e.qa = g->qa;
    e.qb = g->qb;
    e.partials = r.partials;
    e.partials_len = r.len;
    e.sc = r.sc;
    e.counter = r.counter;
    return e;
}

// Set 0: the first 8 max_blocks doubles of the partials buffer and counter[0]; set r > 0: 2 max_blocks
// doubles each after them and counter[32 + r].
RedSet red_set(pbm_grid* g, int rset) {
    if (rset < 0 || rset >= kRedSets) fail(PBM_EINVAL, "reduction set out of range");
    RedSet r;
    r.sc = g->sc;
    if (rset == 0) {
        r.partials = g->partials;
        r.len = int64_t(8) * g->max_blocks;
        r.counter = &g->sc->counter[0];
    } else {
        r.partials = g->partials + int64_t(8 + 2 * (rset - 1)) * g->max_blocks;
        r.len = int64_t(2) * g->max_blocks;
        r.counter = &g->sc->counter[32 + rset];
    }
    return r;
}

int fine_L(const pbm_grid* g, bool fp32, bool op_s) {
    const int L = g->fineL[fp32 ? 1 : 0][op_s ? 1 : 0];
    return L > 0 ? L : fine_chunk(g->L[0].g);
}

template <class T>
void cols_fine(pbm_grid* g, const T* w, const T* d, const T* what, const T* u, const ApplyArgs& a, cudaStream_t st) {
    ColEnv env = env_of(g, a.rset);
    env.L = fine_L(g, sizeof(T) == 4, d != nullptr);
    cols_fine_env<T>(env, g->L[0].g, g->kehat, w, d, what, u, a, st);
}

// Autotuner of the fine column pass: L trades the balance of columns over the SM sub-partitions
// (short chunks, more threads) against the plane transforms shared inside a chunk (long chunks).
// Each candidate is timed with CUDA events on zeroed inputs (the kernels' cost does not depend on
// the values) and the fastest is kept per (precision, operator). For mixed-precision grids the tile
// plans of the single-pass FP32 operator (fused.cu) are timed the same way.
void autotune_fine(pbm_grid* g) {
    const Geom& G = g->L[0].g;
    const int64_t n = G.n(), m = G.m();
    const bool mixed = g->desc.precision == PBM_MIXED;
    PBM_CUDA(cudaMemset(g->kv64[0], 0, sizeof(double) * (n + 1)));
    PBM_CUDA(cudaMemset(g->w64, 0, sizeof(double) * m));
    PBM_CUDA(cudaMemset(g->d64, 0, sizeof(double) * m));
    PBM_CUDA(cudaMemset(g->what_hat, 0, sizeof(double) * 21 * m));
    if (mixed) {
        PBM_CUDA(cudaMemset(g->kv32[0], 0, sizeof(float) * (n + 1)));
        PBM_CUDA(cudaMemset(g->w32, 0, sizeof(float) * m));
        PBM_CUDA(cudaMemset(g->d32, 0, sizeof(float) * m));
        PBM_CUDA(cudaMemset(g->u32, 0, sizeof(float) * (n + 1)));
    }
    cudaEvent_t e0, e1;
    PBM_CUDA(cudaEventCreate(&e0));
    PBM_CUDA(cudaEventCreate(&e1));
    try {
        for (int p = 0; p < (mixed ? 2 : 1); ++p)
            for (int op = 0; op < 2; ++op) {
                ApplyArgs a{};
                a.x = p ? (const void*)g->kv32[0] : (const void*)g->kv64[0];
                a.y = p ? (void*)g->kv32[1] : (void*)g->kv64[1];
                a.mode = EPI_APPLY;
                a.with_alpha = op == 1;
                a.dot_slot = -1;
                float best = 3.4e38f;
                int bestL = 0;
                for (int L = 1; L <= 8; L *= 2) {
                    if (L > 1 && L > G.nz) break;
                    g->fineL[p][op] = L;
                    for (int rep = 0; rep < 4; ++rep) {
                        if (rep == 1) PBM_CUDA(cudaEventRecord(e0, 0));
                        if (p)
                            cols_fine<float>(g, g->w32, op ? g->d32 : nullptr, nullptr, op ? g->u32 : nullptr, a, 0);
                        else
                            cols_fine<double>(g, g->w64, op ? g->d64 : nullptr, op ? g->what_hat : nullptr, nullptr, a,
                                              0);
                    }
                    PBM_CUDA(cudaEventRecord(e1, 0));
                    PBM_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.0f;
                    PBM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) {
                        best = ms;
                        bestL = L;
                    }
                }
                g->fineL[p][op] = bestL;
            }
        // tile plan of the single-pass FP32 operator
        if (mixed)
            for (int op = 0; op < 2; ++op) {
                ApplyArgs a{};
                a.x = g->kv32[0];
                a.y = g->kv32[1];
                a.mode = EPI_APPLY;
                a.with_alpha = op == 1;
                a.dot_slot = -1;
                float best = 3.4e38f;
                int bestP = 0;
                for (int c = 0; c < fused_num_plans(); ++c) {
                    const FusedPlan fp = fused_plan(G, c, op == 1);
                    for (int rep = 0; rep < 4; ++rep) {
                        if (rep == 1) PBM_CUDA(cudaEventRecord(e0, 0));
                        fused_fine_f32(fp, red_set(g, 0), G, g->kehat, g->tc, g->w32, op ? g->d32 : nullptr,
                                       op ? g->u32 : nullptr, a, 0);
                    }
                    PBM_CUDA(cudaEventRecord(e1, 0));
                    PBM_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.0f;
                    PBM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) {
                        best = ms;
                        bestP = c;
                    }
                }
                g->fusedP[op] = bestP;
            }
        // FP32 coarse operator per level that is ever applied: the two passes with eight threads per
        // element (-1) or one (-2), or a plan of the single pass. Levels of 32768 elements or more
        // time only the two-pass forms: their element matrices (1.2 KB per element) dominate and the
        // single pass reads those of its tile halos twice.
        if (mixed)
            for (int k = 1; k + 1 < g->levels; ++k) {
                const Level& L = g->L[k];
                const int last = L.g.m() >= 32768 ? 0 : fused_coarse_num_plans();
                PBM_CUDA(cudaMemset(L.A32, 0, sizeof(float) * NTRI * L.g.m()));
                PBM_CUDA(cudaMemset(L.bord32, 0, sizeof(float) * (L.g.n() + 1)));
                for (int op = 0; op < 2; ++op) {
                    ApplyArgs a{};
                    a.x = g->kv32[0];
                    a.y = g->kv32[1];
                    a.mode = EPI_APPLY;
                    a.with_alpha = op == 1;
                    a.dot_slot = -1;
                    float best = 3.4e38f;
                    int bestP = -1;
                    for (int c = -2; c < last; ++c) {
                        for (int rep = 0; rep < 4; ++rep) {
                            if (rep == 1) PBM_CUDA(cudaEventRecord(e0, 0));
                            if (c < 0)
                                cols_coarse<float>(g, k, L.A32, L.bord32, a, 0, c == -2);
                            else
                                fused_coarse_f32(fused_coarse_plan(L.g, c), red_set(g, 0), L.g, L.A32, L.bord32,
                                                 &g->sc->salpha, a, 0);
                        }
                        PBM_CUDA(cudaEventRecord(e1, 0));
                        PBM_CUDA(cudaEventSynchronize(e1));
                        float ms = 0.0f;
                        PBM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        if (ms < best) {
                            best = ms;
                            bestP = c;
                        }
                    }
                    g->coarseP[op][k] = bestP;
                }
            }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

template <class T>
ColArgs<T> make_coarse_args(const ColEnv& env, const Geom& G, const T* A, const void* x, int* blocks_out) {
    ColArgs<T> P{};
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.support = G.support;
    P.L = 1;
    P.nchunk = G.nz;
    P.n = G.n();
    P.m = G.m();
    P.ncol = int64_t(G.nx) * G.ny;
    P.x = (const T*)x;
    P.A = A;
    P.QA = (T*)env.qa;
    P.QB = (T*)env.qb;
    *blocks_out = int((8 * P.m + CB - 1) / CB);
    return P;
}

template <class T>
void cols_coarse(pbm_grid* g, int k, const T* A, const T* bord, const ApplyArgs& a, cudaStream_t st,
                 bool per_element) {
    const Geom& G = g->L[k].g;
    ColEnv env = env_of(g, a.rset);
    if (g->L[k].qa) {
        env.qa = g->L[k].qa;
        env.qb = g->L[k].qb;
    }
    int blocks = 0;
    const ColArgs<T> P = make_coarse_args<T>(env, G, A, a.x, &blocks);
    if (per_element)
        launch_pdl(k_cols_coarse_e<T>, dim3(unsigned((P.m + CB - 1) / CB)), dim3(CB), 0, st, P);
    else
        launch_pdl(k_cols_coarse<T>, dim3(blocks), dim3(CB), 0, st, P);
    PBM_LAUNCH("coarse column pass");
    node_pass<T>(env, G, a, 1, bord, &g->sc->salpha, nullptr, 0, 0, st);
}

// ---- batched launches (one launch over the systems of a batch) ----
template <class T>
void launch_cols_fine_b(const ColArgs<T>* dA, const BatchMap& M, int mode, int total_blocks, cudaStream_t st) {
    if (mode == 1) k_cols_fine_b<T, 1><<<total_blocks, CB, 0, st>>>(dA, M);
    else if (mode == 2) k_cols_fine_b<T, 2><<<total_blocks, CB, 0, st>>>(dA, M);
    else k_cols_fine_b<T, 0><<<total_blocks, CB, 0, st>>>(dA, M);
    PBM_LAUNCH("batched fine column pass");
}
template <class T>
void launch_cols_coarse_b(const ColArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st) {
    k_cols_coarse_b<T><<<total_blocks, CB, 0, st>>>(dA, M);
    PBM_LAUNCH("batched coarse column pass");
}
template <class T>
void launch_nodes_b(const NodeArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st) {
    k_nodes_b<T><<<total_blocks, NB2, 0, st>>>(dA, M);
    PBM_LAUNCH("batched node pass");
}
#define PBM_INST_BATCH(T)                                                                                         \
    template void launch_cols_fine_b<T>(const ColArgs<T>*, const BatchMap&, int, int, cudaStream_t);           \
    template void launch_cols_coarse_b<T>(const ColArgs<T>*, const BatchMap&, int, cudaStream_t);              \
    template void launch_nodes_b<T>(const NodeArgs<T>*, const BatchMap&, int, cudaStream_t);                   \
    template ColArgs<T> make_fine_args<T>(const ColEnv&, const Geom&, const KeHat&, const T*, const T*, const T*, \
                                          const T*, const void*, int*);                                         \
    template ColArgs<T> make_coarse_args<T>(const ColEnv&, const Geom&, const T*, const void*, int*);          \
    template NodeArgs<T> make_node_args<T>(const ColEnv&, const Geom&, const ApplyArgs&, int, const T*,         \
                                           const double*, const double*, int, int64_t, int*);
PBM_INST_BATCH(double)
PBM_INST_BATCH(float)
#undef PBM_INST_BATCH

template void cols_fine<double>(pbm_grid*, const double*, const double*, const double*, const double*,
                                const ApplyArgs&, cudaStream_t);
template void cols_fine<float>(pbm_grid*, const float*, const float*, const float*, const float*, const ApplyArgs&,
                               cudaStream_t);
template void cols_coarse<double>(pbm_grid*, int, const double*, const double*, const ApplyArgs&, cudaStream_t, bool);
template void cols_coarse<float>(pbm_grid*, int, const float*, const float*, const ApplyArgs&, cudaStream_t, bool);
template void cols_fine_env<double>(const ColEnv&, const Geom&, const KeHat&, const double*, const double*,
                                    const double*, const double*, const ApplyArgs&, cudaStream_t);

// ------------------------------------------------------------------------------------------------
// W_e = Khat H u_e (21 coefficients per element, FP64) for the fine S pass
// ------------------------------------------------------------------------------------------------
__global__ void k_what_hat(int nx, int ny, int nz, int support, const double* __restrict__ u,
                           double* __restrict__ wh, KeHatT<double> K) {
    const int64_t m = int64_t(nx) * ny * nz;
    const int64_t sxn = nx + 1, sxy = int64_t(nx + 1) * (ny + 1);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(e % nx), j = int((e / nx) % ny), k = int(e / (int64_t(nx) * ny));
        double U[3][8], W[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + (a >> 2);
            const bool fx = node_fixed(support, nx, ny, nz, ii, jj, kk);
            const int64_t nd = 3 * (ii + sxn * jj + sxy * kk);
#pragma unroll
            for (int c = 0; c < 3; ++c) U[c][a] = fx ? 0.0 : u[nd + c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) wht_fwd(U[c]);
        khat_apply(K, U, W);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 1; q < 8; ++q) wh[int64_t(7 * c + q - 1) * m + e] = W[c][q];
    }
}

void launch_what_hat(pbm_grid* g, cudaStream_t st) {
    const Geom& G = g->L[0].g;
    KeHatT<double> K;
    fill_khat_t(K, g->kehat);
    const int64_t m = G.m();
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((m + 127) / 128, num_sms() * 16)));
    k_what_hat<<<blocks, 128, 0, st>>>(G.nx, G.ny, G.nz, G.support, g->u64, g->what_hat, K);
    PBM_LAUNCH("what hat");
}

}  // namespace pbm
