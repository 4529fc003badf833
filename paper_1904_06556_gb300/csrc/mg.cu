// Grid transfers and coarse operators of the geometric multigrid V-cycle (Section 5.1, 5.2).
//
//   * prolongation P: 27-point trilinear interpolation from a coarse node grid to its 8-way
//     refinement (a fine node at (I, J, K) takes, per direction, coarse node I/2 if I is even and
//     the mean of (I-1)/2 and (I+1)/2 if I is odd); restriction is P^T; supported dofs are masked
//     on both sides; the extra unknown alpha is transferred by the identity.
//   * coarse operators: Galerkin A_{k-1} = P^T A_k P, element by element. A coarse element's
//     matrix is the sum over its 8 children c of P_c^T A_c P_c, P_c the 24 x 24 interpolation from
//     the coarse element's nodes to child c's nodes. On the first coarse level the fine element
//     matrix is rho'_c K_e + d_c w_c w_c^T (w_c = K_e u_c), so the coarse matrix is
//     sum_c rho'_c G_c + sum_c d_c (P_c^T w_c)(P_c^T w_c)^T with the 8 fixed G_c = P_c^T K_e P_c.
//     The coarse alpha border is b_{k-1} = P^T b_k and S_alpha,alpha is unchanged.
//   * coarsest level: the bordered matrix is assembled densely and factorised by Cholesky in one
//     CTA; L^{-1} (a warp per column) and the explicit inverse L^{-T} L^{-1} (a thread per entry)
//     are spread over the GPU; each V-cycle then applies the inverse (a dense mat-vec).
#include "pbm_internal.h"

namespace pbm {

// 1D interpolation weight of coarse local node A (0/1) at fine position s/2 of the coarse cell
__host__ __device__ inline double wt1(int A, int s) {
    if (s == 1) return 0.5;
    if (s == 0) return A == 0 ? 1.0 : 0.0;
    return A == 1 ? 1.0 : 0.0;
}
// P_c[a][A]: child c, child-local node a, coarse-local node A (a product of 0, 1/2 and 1: exact in
// either precision)
template <class T = double>
__host__ __device__ inline T pc_weight(int c, int a, int A) {
    T w = T(1);
    for (int k = 0; k < 3; ++k) w *= T(wt1((A >> k) & 1, ((c >> k) & 1) + ((a >> k) & 1)));
    return w;
}

// ------------------------------------------------------------------------------------------------
// restriction b_c = P^T r_f (+ alpha copy), times `scale`. One thread per (coarse node, component);
// the 27 weights 1/2^(number of odd offsets) are compile-time constants of the unrolled loops.
// ------------------------------------------------------------------------------------------------
// With xfirst given, the same pass also writes the coarse level's first damped-Jacobi sweep from
// zero, xfirst = omega D^{-1} b_c (idiag = D^{-1} of the coarse level, omega its device weight).

template <class T>
__device__ __forceinline__ void restrict_body(const RestrictArgs<T>& P, unsigned blk, unsigned nblk) {
    const int nxf = P.nxf, nyf = P.nyf, nzf = P.nzf, support = P.support, with_alpha = P.with_alpha;
    const T* __restrict__ rf = P.rf;
    T* __restrict__ bc = P.bc;
    T* __restrict__ xfirst = P.xfirst;
    const T* __restrict__ idiag = P.idiag;
    const double scale = P.scale;
    const double* om = P.om;
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const unsigned nnc = unsigned(nxc + 1) * unsigned(nyc + 1) * unsigned(nzc + 1);
    const int64_t sxf = nxf + 1, sxyf = int64_t(nxf + 1) * (nyf + 1);
    const double w_first = xfirst ? *om : 0.0;
    for (unsigned t = blk * blockDim.x + threadIdx.x; t < 3 * nnc; t += nblk * blockDim.x) {
        const unsigned cn = t / 3u;
        const int c = int(t - 3u * cn);
        const unsigned r = cn / unsigned(nxc + 1);
        const int I = int(cn - r * unsigned(nxc + 1));
        const int J = int(r % unsigned(nyc + 1));
        const int K = int(r / unsigned(nyc + 1));
        // the 27 fine values first (clamped, always valid addresses: the loads do not wait on each
        // other), then the sum over the unmasked ones in a fixed order
        const bool cfix = node_fixed(support, nxc, nyc, nzc, I, J, K);
        T v[27];
        bool ok[27];
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int o = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
                    const int kf = 2 * K + dz, jf = 2 * J + dy, if_ = 2 * I + dx;
                    const bool in = if_ >= 0 && if_ <= nxf && jf >= 0 && jf <= nyf && kf >= 0 && kf <= nzf;
                    ok[o] = in && !cfix && !node_fixed(support, nxf, nyf, nzf, if_, jf, kf);
                    const int ci = min(max(if_, 0), nxf), cj = min(max(jf, 0), nyf), ck = min(max(kf, 0), nzf);
                    v[o] = rf[3 * (ci + sxf * cj + sxyf * ck) + c];
                }
        T acc = T(0);   // accumulated in the vector type (no FP64 work per entry for FP32)
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int o = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
                    const T w = T((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
                    if (ok[o]) acc += w * v[o];
                }
        const T bv = T(scale) * acc;
        bc[t] = bv;
        if (xfirst) xfirst[t] = T(w_first) * (bv * idiag[t]);
    }
    if (with_alpha && blk == 0 && threadIdx.x == 0) {
        const int64_t nf = 3 * int64_t(nxf + 1) * (nyf + 1) * (nzf + 1);
        const T bv = T(scale * double(rf[nf]));
        bc[3 * int64_t(nnc)] = bv;
        if (xfirst) xfirst[3 * int64_t(nnc)] = T(w_first) * (bv * idiag[3 * int64_t(nnc)]);
    }
}

template <class T>
__global__ void k_restrict(RestrictArgs<T> P) {
    pdl_wait();
    pdl_launch_if_small();
    restrict_body<T>(P, blockIdx.x, gridDim.x);
}
template <class T>
__global__ void k_restrict_b(const RestrictArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    restrict_body<T>(A[s], blockIdx.x - M.first[s], M.first[s + 1] - M.first[s]);
}

void launch_restrict(pbm_grid* g, int k, bool fp32, const void* rf, void* bc, bool with_alpha, double scale,
                     cudaStream_t st, void* xfirst) {
    // k: the fine level of the pair (k -> k+1)
    const Geom& F = g->L[k].g;
    Level& C = g->L[k + 1];
    const int64_t nt = 3 * C.g.nnode();
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((nt + 127) / 128, num_sms() * 16)));
    const double* om = &g->sc->mr[16 + k + 1];
    if (fp32)
        launch_pdl(k_restrict<float>, dim3(blocks), dim3(128), 0, st, RestrictArgs<float>{F.nx, F.ny, F.nz, F.support, with_alpha ? 1 : 0,
                                                                      (const float*)rf, (float*)bc, scale,
                                                                      (float*)xfirst, C.idiag32, om});
    else
        launch_pdl(k_restrict<double>, dim3(blocks), dim3(128), 0, st, RestrictArgs<double>{F.nx, F.ny, F.nz, F.support,
                                                                        with_alpha ? 1 : 0, (const double*)rf,
                                                                        (double*)bc, scale, (double*)xfirst,
                                                                        C.idiag64, om});
    PBM_LAUNCH("restrict");
}

// ------------------------------------------------------------------------------------------------
// prolongation x_f += P x_c (+ alpha). One thread per (fine node, component): the up to 8 coarse
// parents share the weight 1/2^(number of odd fine coordinates), built from its exponent bits.
// ------------------------------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ void prolong_body(const ProlongArgs<T>& P, unsigned blk, unsigned nblk) {
    const int nxf = P.nxf, nyf = P.nyf, nzf = P.nzf, support = P.support, with_alpha = P.with_alpha;
    const T* __restrict__ xc = P.xc;
    T* __restrict__ xf = P.xf;
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t nnf = int64_t(nxf + 1) * (nyf + 1) * (nzf + 1);
    const int64_t sxc = nxc + 1, sxyc = int64_t(nxc + 1) * (nyc + 1);
    for (unsigned t = blk * blockDim.x + threadIdx.x; t < 3u * unsigned(nnf); t += nblk * blockDim.x) {
        const unsigned fn = t / 3u;
        const int c = int(t - 3u * fn);
        const unsigned r = fn / unsigned(nxf + 1);
        const int I = int(fn - r * unsigned(nxf + 1));
        const int J = int(r % unsigned(nyf + 1));
        const int K = int(r / unsigned(nyf + 1));
        if (node_fixed(support, nxf, nyf, nzf, I, J, K)) continue;
        // parents per direction: I / 2 for even I, (I - 1) / 2 and (I + 1) / 2 for odd I; every load
        // first, then the sum in the order z, y, x ascending
        const int pi[2] = {I >> 1, (I + 1) >> 1}, pj[2] = {J >> 1, (J + 1) >> 1}, pk[2] = {K >> 1, (K + 1) >> 1};
        const bool oi = (I & 1) != 0, oj = (J & 1) != 0, ok_ = (K & 1) != 0;
        const T xo = xf[t];
        T v[8];
        bool ok[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
            const int ic = pi[bx], jc = pj[by], kc = pk[bz];
            ok[b] = (!bx || oi) && (!by || oj) && (!bz || ok_) && !node_fixed(support, nxc, nyc, nzc, ic, jc, kc);
            v[b] = xc[3 * (ic + sxc * jc + sxyc * kc) + c];
        }
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (ok[b]) acc += v[b];
        const int nodd = (I & 1) + (J & 1) + (K & 1);
        const T w = T(__longlong_as_double(static_cast<long long>(1023 - nodd) << 52));  // 2^-nodd, exact
        xf[t] = xo + w * acc;
    }
    if (with_alpha && blk == 0 && threadIdx.x == 0) {
        const int64_t nc = 3 * int64_t(nxc + 1) * (nyc + 1) * (nzc + 1);
        xf[3 * nnf] += xc[nc];
    }
}

template <class T>
__global__ void k_prolong_add(ProlongArgs<T> P) {
    pdl_wait();
    pdl_launch_if_small();
    prolong_body<T>(P, blockIdx.x, gridDim.x);
}
template <class T>
__global__ void k_prolong_add_b(const ProlongArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    prolong_body<T>(A[s], blockIdx.x - M.first[s], M.first[s + 1] - M.first[s]);
}

void launch_prolong_add(pbm_grid* g, int k, bool fp32, const void* xc, void* xf, bool with_alpha, cudaStream_t st) {
    const Geom& F = g->L[k].g;
    const int64_t nt = 3 * F.nnode();
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((nt + 255) / 256, num_sms() * 16)));
    if (fp32)
        launch_pdl(k_prolong_add<float>, dim3(blocks), dim3(256), 0, st, ProlongArgs<float>{F.nx, F.ny, F.nz, F.support,
                                                                        with_alpha ? 1 : 0, (const float*)xc,
                                                                        (float*)xf});
    else
        launch_pdl(k_prolong_add<double>, dim3(blocks), dim3(256), 0, st, ProlongArgs<double>{F.nx, F.ny, F.nz, F.support,
                                                                          with_alpha ? 1 : 0, (const double*)xc,
                                                                          (double*)xf});
    PBM_LAUNCH("prolong");
}

// ------------------------------------------------------------------------------------------------
// what[i][e] = (P_c^T K_e u_e)[i] for every fine element e (child c = parities of its indices)
// ------------------------------------------------------------------------------------------------
template <class T>
__global__ void k_build_what(int nx, int ny, int nz, int support, const T* __restrict__ u, T* __restrict__ what,
                             KeHatT<T> K) {
    const int64_t m = int64_t(nx) * ny * nz;
    const int64_t sxn = nx + 1, sxy = int64_t(nx + 1) * (ny + 1);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(e % nx);
        const int j = int((e / nx) % ny);
        const int k = int(e / (int64_t(nx) * ny));
        const int c = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
        T U[3][8], W[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + ((a >> 2) & 1);
            const bool fx = node_fixed(support, nx, ny, nz, ii, jj, kk);
            const int64_t nd = 3 * (ii + sxn * jj + sxy * kk);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) U[cc][a] = fx ? T(0) : u[nd + cc];
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) wht_fwd(U[cc]);
        khat_apply(K, U, W);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) wht_out(W[cc]);
        // W[cc][a] = (K_e u_e)[3a + cc]; project with P_c^T
#pragma unroll
        for (int A = 0; A < 8; ++A) {
            T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const T p = pc_weight<T>(c, a, A);
                s0 += p * W[0][a];
                s1 += p * W[1][a];
                s2 += p * W[2][a];
            }
            what[(3 * A) * m + e] = s0;
            what[(3 * A + 1) * m + e] = s1;
            what[(3 * A + 2) * m + e] = s2;
        }
    }
}

// fp32: the table in FP32 from the FP32 copy of u, into the first half of the FP64 table's buffer
// (mixed grids: it only feeds the FP32 Galerkin chain of the set-up)
void launch_build_what(pbm_grid* g, cudaStream_t st, bool fp32) {
    const Geom& G = g->L[0].g;
    const int64_t m = G.m();
    const int blocks = int(std::min<int64_t>((m + 127) / 128, num_sms() * 16));
    if (fp32) {
        KeHatT<float> K;
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < 8; ++q) K.dg[c][q] = float(g->kehat.dg[c][q]);
        for (int b = 0; b < 2; ++b) {
            K.lam4[b] = float(g->kehat.lam4[b]);
            K.mu4[b] = float(g->kehat.mu4[b]);
        }
        k_build_what<float><<<blocks, 128, 0, st>>>(G.nx, G.ny, G.nz, G.support, g->u32, (float*)g->what, K);
    } else {
        KeHatT<double> K;
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < 8; ++q) K.dg[c][q] = g->kehat.dg[c][q];
        for (int b = 0; b < 2; ++b) {
            K.lam4[b] = g->kehat.lam4[b];
            K.mu4[b] = g->kehat.mu4[b];
        }
        k_build_what<double><<<blocks, 128, 0, st>>>(G.nx, G.ny, G.nz, G.support, g->u64, g->what, K);
    }
    PBM_LAUNCH("build what");
}

// ------------------------------------------------------------------------------------------------
// level 1 element matrices: sum_c w_c G_c (+ d_c what_c what_c^T); one thread per (coarse element E,
// row i) forms the row's entries (i, j), j >= i: the children's weights and d_c what_i,c are loaded
// (formed) once per thread, so every entry costs two FMAs per child and one load of what_j,c.
// Warps hold 32 consecutive elements of one row: every load and store is coalesced.
// ------------------------------------------------------------------------------------------------
template <class T>
__global__ void k_build_level1(int nxf, int nyf, int nzf, const T* __restrict__ w, const T* __restrict__ d,
                               const T* __restrict__ what, const T* __restrict__ G, T* __restrict__ A) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t mc = int64_t(nxc) * nyc * nzc, mf = int64_t(nxf) * nyf * nzf;
    const int ii = blockIdx.y;
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < mc; E += int64_t(gridDim.x) * blockDim.x) {
        const int I = int(E % nxc);
        const int J = int((E / nxc) % nyc);
        const int K = int(E / (int64_t(nxc) * nyc));
        int64_t e[8];
        T wc[8], dwi[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            e[c] = (2 * I + (c & 1)) + int64_t(nxf) * ((2 * J + ((c >> 1) & 1)) + int64_t(nyf) * (2 * K + (c >> 2)));
            wc[c] = w[e[c]];
            dwi[c] = d ? d[e[c]] * what[ii * mf + e[c]] : T(0);
        }
        for (int jj = ii; jj < 24; ++jj) {
            const int t = tri_index(ii, jj);
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                acc += wc[c] * G[c * NTRI + t];
                if (d) acc += dwi[c] * what[jj * mf + e[c]];
            }
            A[t * mc + E] = acc;
        }
    }
}

// fp32 (mixed grids): from the FP32 weights and table into the FP32 matrices the V-cycle applies
void launch_build_level1(pbm_grid* g, bool op_s, cudaStream_t st, bool fp32) {
    const Geom& F = g->L[0].g;
    const int64_t mc = g->L[1].g.m();
    dim3 grid(unsigned(std::max<int64_t>(1, std::min<int64_t>((mc + 127) / 128, 1024))), 24);
    if (fp32)
        k_build_level1<float><<<grid, 128, 0, st>>>(F.nx, F.ny, F.nz, op_s ? g->w32 : g->rho32,
                                                    op_s ? g->d32 : nullptr, (const float*)g->what, g->G32,
                                                    g->L[1].A32);
    else
        k_build_level1<double><<<grid, 128, 0, st>>>(F.nx, F.ny, F.nz, op_s ? g->w64 : g->rho,
                                                     op_s ? g->d64 : nullptr, g->what, g->G_dev, g->L[1].A64);
    PBM_LAUNCH("build level1");
}

// ------------------------------------------------------------------------------------------------
// level k+1 from level k: sum_c P_c^T A_c P_c
//
// P_c acts on the node index only and is a tensor product of one 2 x 2 interpolation per axis
// (child bit 0: rows (1, 0), (1/2, 1/2); child bit 1: rows (1/2, 1/2), (0, 1)). So each 8 x 8 block
// A_ij (displacement components i, j) of a child matrix is transformed on its own, B_ij = P^T A_ij
// P, by three one-dimensional passes on each side. A group of 8 lanes holds the 8 children of one
// coarse element and one block (i <= j); the lanes sum their results with shuffles and each writes
// 8 of the 64 entries into the coarse upper triangle (every triangle entry is written once: an
// entry (r, s), r <= s, belongs to block (r % 3, s % 3) if r % 3 <= s % 3, else to the transposed
// position of block (s % 3, r % 3)).
// ------------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void interp_pair(T& v0, T& v1, int cb) {
    const T h = T(0.5) * (cb ? v0 : v1);
    const T sum = (cb ? v1 : v0) + h;
    v0 = cb ? h : sum;
    v1 = cb ? sum : h;
}

template <class T>
__device__ __forceinline__ void interp8(T (&v)[8], int c) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int cb = (c >> ax) & 1;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (!((b >> ax) & 1)) interp_pair(v[b], v[b | (1 << ax)], cb);
    }
}

template <class T>
__global__ void __launch_bounds__(128) k_build_coarser(int nxf, int nyf, int nzf, const T* __restrict__ Af,
                                                       T* __restrict__ Ac) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t mc = int64_t(nxc) * nyc * nzc, mf = int64_t(nxf) * nyf * nzf;
    const int64_t tid = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int c = int(tid & 7);
    const int64_t grp = tid >> 3;
    const int blk = int(grp % 6);
    int64_t E = grp / 6;
    const bool live = E < mc;
    if (!live) E = mc - 1;   // keep the lane in the shuffles
    const int bi = blk < 3 ? 0 : (blk < 5 ? 1 : 2);
    const int bj = blk < 3 ? blk : (blk < 5 ? blk - 2 : 2);
    const int ex = int(E % nxc), ey = int((E / nxc) % nyc), ez = int(E / (int64_t(nxc) * nyc));
    const int64_t e = (2 * ex + (c & 1)) + int64_t(nxf) * ((2 * ey + ((c >> 1) & 1)) + int64_t(nyf) * (2 * ez + (c >> 2)));
    T M[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int r = 3 * a + bi, q = 3 * b + bj;
            const int t = r <= q ? tri_index(r, q) : tri_index(q, r);
            M[a][b] = Af[int64_t(t) * mf + e];
        }
    // right: rows, left: columns
#pragma unroll
    for (int a = 0; a < 8; ++a) interp8(M[a], c);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        T col[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) col[a] = M[a][b];
        interp8(col, c);
#pragma unroll
        for (int a = 0; a < 8; ++a) M[a][b] = col[a];
    }
    // sum over the 8 children (lanes of the group), fixed order
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            T v = M[a][b];
            v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
            M[a][b] = v;
        }
    if (!live) return;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        // lane c writes row A = a of the block when a == c (8 entries each)
        if (a != c) continue;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (bi == bj && b < a) continue;
            const int r = 3 * a + bi, q = 3 * b + bj;
            const int t = r <= q ? tri_index(r, q) : tri_index(q, r);
            Ac[int64_t(t) * mc + E] = M[a][b];
        }
    }
}

void launch_build_coarser(pbm_grid* g, int k, cudaStream_t st, bool fp32) {
    const Geom& F = g->L[k].g;
    const int64_t mc = g->L[k + 1].g.m();
    const int blocks = int((mc * 48 + 127) / 128);
    if (fp32)
        k_build_coarser<float><<<blocks, 128, 0, st>>>(F.nx, F.ny, F.nz, g->L[k].A32, g->L[k + 1].A32);
    else
        k_build_coarser<double><<<blocks, 128, 0, st>>>(F.nx, F.ny, F.nz, g->L[k].A64, g->L[k + 1].A64);
    PBM_LAUNCH("build coarser");
}

// FP32 copies of level k's alpha border and, when built in FP64, its matrices (mixed grids)
void launch_coarse_to_f32(pbm_grid* g, int k, cudaStream_t st, bool matrices) {
    Level& L = g->L[k];
    if (matrices && L.A32) launch_cast(L.A64, false, L.A32, true, int64_t(NTRI) * L.g.m(), st);
    if (L.bord32) launch_cast(L.bord64, false, L.bord32, true, L.g.n(), st);
}

// FP64 matrices of level k from its FP32 ones (the coarsest level of a mixed grid, for its FP64
// Cholesky factorisation: the factor then inverts exactly the matrix the FP32 V-cycle restricts to)
void launch_coarse_to_f64(pbm_grid* g, int k, cudaStream_t st) {
    Level& L = g->L[k];
    launch_cast(L.A32, true, L.A64, false, int64_t(NTRI) * L.g.m(), st);
}

// ------------------------------------------------------------------------------------------------
// coarsest level: dense assembly and Cholesky (one CTA), then L^{-1} (a warp per column) and the
// explicit inverse L^{-T} L^{-1} (one thread per entry) spread over many SMs
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_coarsest_factor(int nx, int ny, int nz, int support, const double* __restrict__ A,
                                  const double* __restrict__ bord, double s_alpha, int op_s, double* __restrict__ Mg,
                                  double* __restrict__ Dinv, int* flag, int use_smem) {
    extern __shared__ double smem[];
    double* M = use_smem ? smem : Mg;   // the factorisation runs in shared memory when N^2 fits
    const int64_t m = int64_t(nx) * ny * nz;
    const int n = 3 * (nx + 1) * (ny + 1) * (nz + 1);
    const int N = n + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int i = tid; i < N * N; i += nt) M[i] = 0.0;
    __syncthreads();
    const int sx = nx + 1, sxy = (nx + 1) * (ny + 1);
    // assemble element by element in a fixed order (entries of one element hit distinct cells)
    for (int64_t e = 0; e < m; ++e) {
        const int i = int(e % nx), j = int((e / nx) % ny), k = int(e / (int64_t(nx) * ny));
        for (int t = tid; t < NTRI; t += nt) {
            int r = 0, c = 0;
            // decode t -> (r, c)
            {
                int acc = 0;
                for (r = 0; r < 24; ++r) {
                    if (t < acc + (24 - r)) break;
                    acc += 24 - r;
                }
                c = r + (t - acc);
            }
            const int ar = r / 3, cr = r % 3, ac = c / 3, cc = c % 3;
            const int nr = (i + (ar & 1)) + sx * (j + ((ar >> 1) & 1)) + sxy * (k + (ar >> 2));
            const int nc2 = (i + (ac & 1)) + sx * (j + ((ac >> 1) & 1)) + sxy * (k + (ac >> 2));
            const int R = 3 * nr + cr, C = 3 * nc2 + cc;
            const double v = A[t * m + e];
            M[R * N + C] += v;
            if (R != C) M[C * N + R] += v;
        }
        __syncthreads();
    }
    // supports, border
    for (int R = tid; R < n; R += nt) {
        const int nd = R / 3;
        const int ii = nd % sx, jj = (nd / sx) % (ny + 1), kk = nd / sxy;
        const bool fx = node_fixed(support, nx, ny, nz, ii, jj, kk);
        if (fx) {
            for (int C = 0; C < N; ++C) {
                M[R * N + C] = 0.0;
                M[C * N + R] = 0.0;
            }
        }
        M[R * N + n] = M[n * N + R] = (op_s && !fx) ? bord[R] : 0.0;
    }
    __syncthreads();
    for (int R = tid; R < n; R += nt) {
        const int nd = R / 3;
        const int ii = nd % sx, jj = (nd / sx) % (ny + 1), kk = nd / sxy;
        if (node_fixed(support, nx, ny, nz, ii, jj, kk)) M[R * N + R] = 1.0;
    }
    if (tid == 0) M[n * N + n] = op_s ? s_alpha : 1.0;
    __syncthreads();
    // Cholesky (lower, in place); the reciprocal of each pivot replaces N - j divisions
    __shared__ double ipiv;
    for (int j = 0; j < N; ++j) {
        if (tid == 0) {
            const double a = M[j * N + j];
            if (!(a > 0.0)) *flag = 1;
            const double piv = a > 0.0 ? sqrt(a) : 1.0;
            M[j * N + j] = piv;
            ipiv = 1.0 / piv;
        }
        __syncthreads();
        const double ip = ipiv;
        for (int i = j + 1 + tid; i < N; i += nt) M[i * N + j] *= ip;
        __syncthreads();
        // trailing update of the lower triangle: a warp per row, lanes over the columns
        for (int i = j + 1 + wid; i < N; i += nw) {
            const double lij = M[i * N + j];
            for (int k = j + 1 + lane; k <= i; k += 32) M[i * N + k] -= lij * M[k * N + j];
        }
        __syncthreads();
    }
    // reciprocals of the diagonal of L for the substitutions
    for (int i = tid; i < N; i += nt) Dinv[i] = 1.0 / M[i * N + i];
    if (use_smem)
        for (int i = tid; i < N * N; i += nt) Mg[i] = M[i];
}

constexpr int COARSEST_SMEM_N = 160;   // shared-memory factorisation up to N = 160 (200 KB)

// column c of L^{-1} by forward substitution, one warp per column (lanes split the dot products)
__global__ void k_coarsest_linv(int N, const double* __restrict__ M, const double* __restrict__ Dinv,
                                double* __restrict__ Linv) {
    const int lane = threadIdx.x & 31;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= N) return;
    for (int i = 0; i < col; ++i)
        if (lane == 0) Linv[i * N + col] = 0.0;
    for (int i = col; i < N; ++i) {
        double s = 0.0;
        for (int k = col + lane; k < i; k += 32) s += M[i * N + k] * Linv[k * N + col];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double v = ((i == col ? 1.0 : 0.0) - s) * Dinv[i];
        if (lane == 0) Linv[i * N + col] = v;
        __syncwarp();
    }
}

// A^{-1} = L^{-T} L^{-1}: entry (r, c) = sum_{k >= max(r, c)} Linv[k][r] Linv[k][c], symmetric
__global__ void k_coarsest_inv(int N, const double* __restrict__ Linv, double* __restrict__ Inv) {
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (t >= int64_t(N) * N) return;
    const int r = int(t / N), c = int(t % N);
    if (c < r) return;
    double s = 0.0;
    for (int k = c; k < N; ++k) s += Linv[k * N + r] * Linv[k * N + c];
    Inv[r * N + c] = s;
    Inv[c * N + r] = s;
}

void build_coarsest(pbm_grid* g, bool op_s, cudaStream_t st) {
    const int kc = g->levels - 1;
    Level& L = g->L[kc];
    PBM_CUDA(cudaMemsetAsync(&g->sc->flags[0], 0, sizeof(int), st));
    if (kc == 0) fail(PBM_EINVAL, "a single-level hierarchy has no coarse operator (use levels >= 2)");
    const int N = g->nc + 1;
    double* M = g->cwork;
    double* Linv = g->cwork + size_t(N) * N;
    double* Dinv = g->cwork + 2 * size_t(N) * N;
    const bool sm = N <= COARSEST_SMEM_N;
    const size_t smem = sm ? sizeof(double) * size_t(N) * N : 0;
    if (sm) {
        static bool attr_done[64] = {};
        if (!attr_done[g->device & 63]) {
            PBM_CUDA(cudaFuncSetAttribute(k_coarsest_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(sizeof(double) * COARSEST_SMEM_N * COARSEST_SMEM_N)));
            attr_done[g->device & 63] = true;
        }
    }
    k_coarsest_factor<<<1, 1024, smem, st>>>(L.g.nx, L.g.ny, L.g.nz, L.g.support, L.A64, L.bord64, g->s_alpha,
                                             op_s ? 1 : 0, M, Dinv, &g->sc->flags[0], sm ? 1 : 0);
    PBM_LAUNCH("coarsest factor");
    k_coarsest_linv<<<(N * 32 + 127) / 128, 128, 0, st>>>(N, M, Dinv, Linv);
    PBM_LAUNCH("coarsest L inverse");
    k_coarsest_inv<<<int((int64_t(N) * N + 255) / 256), 256, 0, st>>>(N, Linv, g->cinv);
    PBM_LAUNCH("coarsest inverse");
}

// x = Inv b on the coarsest level (warp per row, FP64 accumulation)

template <class T>
__device__ __forceinline__ void coarsest_solve_body(const CoarsestArgs<T>& P, unsigned blk) {
    const int N = P.N, n_vec = P.n_vec;
    const double* __restrict__ Inv = P.Inv;
    const T* __restrict__ b = P.b;
    T* __restrict__ x = P.x;
    const int lane = threadIdx.x & 31;
    const int row = int((blk * blockDim.x + threadIdx.x) >> 5);
    if (row >= n_vec) return;
    double s = 0.0;
    // the lane's terms c = lane, lane + 32, ... in ascending order, eight loads of each operand ahead
    for (int c0 = 0; c0 < n_vec; c0 += 256) {
        double iv[8], bv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + 32 * u + lane;
            const int cc = c < n_vec ? c : 0;
            iv[u] = Inv[row * N + cc];
            bv[u] = double(b[cc]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c0 + 32 * u + lane < n_vec) s += iv[u] * bv[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = T(s);
}

template <class T>
__global__ void k_coarsest_solve(CoarsestArgs<T> P) {
    pdl_wait();
    pdl_launch_if_small();
    coarsest_solve_body<T>(P, blockIdx.x);
}
template <class T>
__global__ void k_coarsest_solve_b(const CoarsestArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    coarsest_solve_body<T>(A[s], blockIdx.x - M.first[s]);
}

void launch_coarsest_solve(pbm_grid* g, bool fp32, const void* b, void* x, bool with_alpha, cudaStream_t st) {
    const int N = g->nc + 1;
    const int nv = with_alpha ? N : N - 1;
    const int blocks = (nv * 32 + 255) / 256;
    if (fp32) launch_pdl(k_coarsest_solve<float>, dim3(blocks), dim3(256), 0, st, CoarsestArgs<float>{N, nv, g->cinv, (const float*)b, (float*)x});
    else launch_pdl(k_coarsest_solve<double>, dim3(blocks), dim3(256), 0, st, CoarsestArgs<double>{N, nv, g->cinv, (const double*)b, (double*)x});
    PBM_LAUNCH("coarsest solve");
}

template <class T>
RestrictArgs<T> make_restrict_args(pbm_grid* g, int k, const void* rf, void* bc, bool with_alpha, double scale,
                                   void* xfirst, int* blocks_out) {
    const Geom& F = g->L[k].g;
    Level& C = g->L[k + 1];
    const int64_t nt = 3 * C.g.nnode();
    *blocks_out = int(std::max<int64_t>(1, std::min<int64_t>((nt + 127) / 128, num_sms() * 16)));
    const T* idiag = sizeof(T) == 4 ? (const T*)(const void*)C.idiag32 : (const T*)(const void*)C.idiag64;
    return RestrictArgs<T>{F.nx, F.ny, F.nz, F.support, with_alpha ? 1 : 0, (const T*)rf, (T*)bc, scale,
                           (T*)xfirst, idiag, &g->sc->mr[16 + k + 1]};
}
template <class T>
ProlongArgs<T> make_prolong_args(pbm_grid* g, int k, const void* xc, void* xf, bool with_alpha, int* blocks_out) {
    const Geom& F = g->L[k].g;
    const int64_t nt = 3 * F.nnode();
    *blocks_out = int(std::max<int64_t>(1, std::min<int64_t>((nt + 255) / 256, num_sms() * 16)));
    return ProlongArgs<T>{F.nx, F.ny, F.nz, F.support, with_alpha ? 1 : 0, (const T*)xc, (T*)xf};
}
template <class T>
CoarsestArgs<T> make_coarsest_args(pbm_grid* g, const void* b, void* x, bool with_alpha, int* blocks_out) {
    const int N = g->nc + 1;
    const int nv = with_alpha ? N : N - 1;
    *blocks_out = (nv * 32 + 255) / 256;
    return CoarsestArgs<T>{N, nv, g->cinv, (const T*)b, (T*)x};
}
template <class T>
void launch_restrict_b(const RestrictArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st) {
    k_restrict_b<T><<<total_blocks, 128, 0, st>>>(dA, M);
    PBM_LAUNCH("batched restrict");
}
template <class T>
void launch_prolong_b(const ProlongArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st) {
    k_prolong_add_b<T><<<total_blocks, 256, 0, st>>>(dA, M);
    PBM_LAUNCH("batched prolong");
}
template <class T>
void launch_coarsest_b(const CoarsestArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st) {
    k_coarsest_solve_b<T><<<total_blocks, 256, 0, st>>>(dA, M);
    PBM_LAUNCH("batched coarsest solve");
}
#define PBM_INST_MG(T)                                                                                          \
    template RestrictArgs<T> make_restrict_args<T>(pbm_grid*, int, const void*, void*, bool, double, void*, int*); \
    template ProlongArgs<T> make_prolong_args<T>(pbm_grid*, int, const void*, void*, bool, int*);               \
    template CoarsestArgs<T> make_coarsest_args<T>(pbm_grid*, const void*, void*, bool, int*);                  \
    template void launch_restrict_b<T>(const RestrictArgs<T>*, const BatchMap&, int, cudaStream_t);             \
    template void launch_prolong_b<T>(const ProlongArgs<T>*, const BatchMap&, int, cudaStream_t);               \
    template void launch_coarsest_b<T>(const CoarsestArgs<T>*, const BatchMap&, int, cudaStream_t);
PBM_INST_MG(double)
PBM_INST_MG(float)
#undef PBM_INST_MG

}  // namespace pbm
