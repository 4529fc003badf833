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
//   * coarsest level: the bordered matrix is assembled densely, factorised by Cholesky in one
//     CTA, and inverted explicitly; each V-cycle then applies the inverse (a dense mat-vec).
#include "pbm_internal.h"

namespace pbm {

// 1D interpolation weight of coarse local node A (0/1) at fine position s/2 of the coarse cell
__host__ __device__ inline double wt1(int A, int s) {
    if (s == 1) return 0.5;
    if (s == 0) return A == 0 ? 1.0 : 0.0;
    return A == 1 ? 1.0 : 0.0;
}
// P_c[a][A]: child c, child-local node a, coarse-local node A
__host__ __device__ inline double pc_weight(int c, int a, int A) {
    double w = 1.0;
    for (int k = 0; k < 3; ++k) w *= wt1((A >> k) & 1, ((c >> k) & 1) + ((a >> k) & 1));
    return w;
}

// ------------------------------------------------------------------------------------------------
// restriction b_c = P^T r_f (+ alpha copy), times `scale`
// ------------------------------------------------------------------------------------------------
template <class T>
__global__ void k_restrict(int nxf, int nyf, int nzf, int support, const T* __restrict__ rf, T* __restrict__ bc,
                           int with_alpha, double scale) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t nnc = int64_t(nxc + 1) * (nyc + 1) * (nzc + 1);
    const int64_t sxf = nxf + 1, sxyf = int64_t(nxf + 1) * (nyf + 1);
    for (int64_t cn = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; cn < nnc; cn += int64_t(gridDim.x) * blockDim.x) {
        const int I = int(cn % (nxc + 1));
        const int J = int((cn / (nxc + 1)) % (nyc + 1));
        const int K = int(cn / (int64_t(nxc + 1) * (nyc + 1)));
        double acc[3] = {0.0, 0.0, 0.0};
        if (!node_fixed(support, nxc, nyc, nzc, I, J, K)) {
            for (int dz = -1; dz <= 1; ++dz) {
                const int kf = 2 * K + dz;
                if (kf < 0 || kf > nzf) continue;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int jf = 2 * J + dy;
                    if (jf < 0 || jf > nyf) continue;
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int if_ = 2 * I + dx;
                        if (if_ < 0 || if_ > nxf) continue;
                        if (node_fixed(support, nxf, nyf, nzf, if_, jf, kf)) continue;
                        const double w = (dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0);
                        const int64_t f = 3 * (if_ + sxf * jf + sxyf * kf);
                        acc[0] += w * double(rf[f]);
                        acc[1] += w * double(rf[f + 1]);
                        acc[2] += w * double(rf[f + 2]);
                    }
                }
            }
        }
        bc[3 * cn] = T(scale * acc[0]);
        bc[3 * cn + 1] = T(scale * acc[1]);
        bc[3 * cn + 2] = T(scale * acc[2]);
    }
    if (with_alpha && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t nf = 3 * int64_t(nxf + 1) * (nyf + 1) * (nzf + 1);
        bc[3 * nnc] = T(scale * double(rf[nf]));
    }
}

void launch_restrict(pbm_grid* g, int k, bool fp32, const void* rf, void* bc, bool with_alpha, double scale,
                     cudaStream_t st) {
    // k: the fine level of the pair (k -> k+1)
    const Geom& F = g->L[k].g;
    const int64_t nnc = g->L[k + 1].g.nnode();
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((nnc + 255) / 256, 152 * 8)));
    if (fp32)
        k_restrict<float><<<blocks, 256, 0, st>>>(F.nx, F.ny, F.nz, F.support, (const float*)rf, (float*)bc,
                                                  with_alpha, scale);
    else
        k_restrict<double><<<blocks, 256, 0, st>>>(F.nx, F.ny, F.nz, F.support, (const double*)rf, (double*)bc,
                                                   with_alpha, scale);
    PBM_LAUNCH("restrict");
}

// ------------------------------------------------------------------------------------------------
// prolongation x_f += P x_c (+ alpha)
// ------------------------------------------------------------------------------------------------
template <class T>
__global__ void k_prolong_add(int nxf, int nyf, int nzf, int support, const T* __restrict__ xc, T* __restrict__ xf,
                              int with_alpha) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t nnf = int64_t(nxf + 1) * (nyf + 1) * (nzf + 1);
    const int64_t sxc = nxc + 1, sxyc = int64_t(nxc + 1) * (nyc + 1);
    for (int64_t fn = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; fn < nnf; fn += int64_t(gridDim.x) * blockDim.x) {
        const int I = int(fn % (nxf + 1));
        const int J = int((fn / (nxf + 1)) % (nyf + 1));
        const int K = int(fn / (int64_t(nxf + 1) * (nyf + 1)));
        if (node_fixed(support, nxf, nyf, nzf, I, J, K)) continue;
        double acc[3] = {0.0, 0.0, 0.0};
        const int i0 = I >> 1, i1 = (I + 1) >> 1, j0 = J >> 1, j1 = (J + 1) >> 1, k0 = K >> 1, k1 = (K + 1) >> 1;
        const double wx = (I & 1) ? 0.5 : 1.0, wy = (J & 1) ? 0.5 : 1.0, wz = (K & 1) ? 0.5 : 1.0;
        for (int kc = k0; kc <= k1; ++kc)
            for (int jc = j0; jc <= j1; ++jc)
                for (int ic = i0; ic <= i1; ++ic) {
                    if (node_fixed(support, nxc, nyc, nzc, ic, jc, kc)) continue;
                    const double w = wx * wy * wz;
                    const int64_t c = 3 * (ic + sxc * jc + sxyc * kc);
                    acc[0] += w * double(xc[c]);
                    acc[1] += w * double(xc[c + 1]);
                    acc[2] += w * double(xc[c + 2]);
                }
        xf[3 * fn] += T(acc[0]);
        xf[3 * fn + 1] += T(acc[1]);
        xf[3 * fn + 2] += T(acc[2]);
    }
    if (with_alpha && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t nc = 3 * int64_t(nxc + 1) * (nyc + 1) * (nzc + 1);
        xf[3 * nnf] += xc[nc];
    }
}

void launch_prolong_add(pbm_grid* g, int k, bool fp32, const void* xc, void* xf, bool with_alpha, cudaStream_t st) {
    const Geom& F = g->L[k].g;
    const int64_t nnf = F.nnode();
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((nnf + 255) / 256, 152 * 8)));
    if (fp32)
        k_prolong_add<float><<<blocks, 256, 0, st>>>(F.nx, F.ny, F.nz, F.support, (const float*)xc, (float*)xf,
                                                     with_alpha);
    else
        k_prolong_add<double><<<blocks, 256, 0, st>>>(F.nx, F.ny, F.nz, F.support, (const double*)xc, (double*)xf,
                                                      with_alpha);
    PBM_LAUNCH("prolong");
}

// ------------------------------------------------------------------------------------------------
// what[i][e] = (P_c^T K_e u_e)[i] for every fine element e (child c = parities of its indices)
// ------------------------------------------------------------------------------------------------
__global__ void k_build_what(int nx, int ny, int nz, int support, const double* __restrict__ u,
                             double* __restrict__ what, KeHatT<double> K) {
    const int64_t m = int64_t(nx) * ny * nz;
    const int64_t sxn = nx + 1, sxy = int64_t(nx + 1) * (ny + 1);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(e % nx);
        const int j = int((e / nx) % ny);
        const int k = int(e / (int64_t(nx) * ny));
        const int c = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
        double U[3][8], W[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + ((a >> 2) & 1);
            const bool fx = node_fixed(support, nx, ny, nz, ii, jj, kk);
            const int64_t nd = 3 * (ii + sxn * jj + sxy * kk);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) U[cc][a] = fx ? 0.0 : u[nd + cc];
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) wht_fwd(U[cc]);
        khat_apply(K, U, W);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) wht_out(W[cc]);
        // W[cc][a] = (K_e u_e)[3a + cc]; project with P_c^T
#pragma unroll
        for (int A = 0; A < 8; ++A) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const double p = pc_weight(c, a, A);
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

void launch_build_what(pbm_grid* g, cudaStream_t st) {
    const Geom& G = g->L[0].g;
    KeHatT<double> K;
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 8; ++q) K.dg[c][q] = g->kehat.dg[c][q];
    for (int b = 0; b < 2; ++b) {
        K.lam4[b] = g->kehat.lam4[b];
        K.mu4[b] = g->kehat.mu4[b];
    }
    const int64_t m = G.m();
    const int blocks = int(std::min<int64_t>((m + 127) / 128, 152 * 16));
    k_build_what<<<blocks, 128, 0, st>>>(G.nx, G.ny, G.nz, G.support, g->u64, g->what, K);
    PBM_LAUNCH("build what");
}

// ------------------------------------------------------------------------------------------------
// level 1 element matrices: sum_c w_c G_c (+ d_c what_c what_c^T); one thread per (element, entry)
// ------------------------------------------------------------------------------------------------
__constant__ int c_tri_i[NTRI];
__constant__ int c_tri_j[NTRI];

__global__ void k_build_level1(int nxf, int nyf, int nzf, const double* __restrict__ w, const double* __restrict__ d,
                               const double* __restrict__ what, const double* __restrict__ G, double* __restrict__ A) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t mc = int64_t(nxc) * nyc * nzc, mf = int64_t(nxf) * nyf * nzf;
    const int t = blockIdx.y;
    const int ii = c_tri_i[t], jj = c_tri_j[t];
    double Gc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) Gc[c] = G[c * NTRI + t];
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < mc; E += int64_t(gridDim.x) * blockDim.x) {
        const int I = int(E % nxc);
        const int J = int((E / nxc) % nyc);
        const int K = int(E / (int64_t(nxc) * nyc));
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t e = (2 * I + (c & 1)) + int64_t(nxf) * ((2 * J + ((c >> 1) & 1)) + int64_t(nyf) * (2 * K + (c >> 2)));
            acc += w[e] * Gc[c];
            if (d) acc += d[e] * what[ii * mf + e] * what[jj * mf + e];
        }
        A[t * mc + E] = acc;
    }
}

void launch_build_level1(pbm_grid* g, bool op_s, cudaStream_t st) {
    const Geom& F = g->L[0].g;
    const int64_t mc = g->L[1].g.m();
    dim3 grid(unsigned(std::max<int64_t>(1, std::min<int64_t>((mc + 127) / 128, 64))), NTRI);
    k_build_level1<<<grid, 128, 0, st>>>(F.nx, F.ny, F.nz, op_s ? g->w64 : g->rho, op_s ? g->d64 : nullptr, g->what, g->G_dev,
                                          g->L[1].A64);
    PBM_LAUNCH("build level1");
}

// ------------------------------------------------------------------------------------------------
// level k+1 from level k: sum_c P_c^T A_c P_c
// ------------------------------------------------------------------------------------------------
__global__ void k_build_coarser(int nxf, int nyf, int nzf, const double* __restrict__ Af, double* __restrict__ Ac) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const int64_t mc = int64_t(nxc) * nyc * nzc, mf = int64_t(nxf) * nyf * nzf;
    const int t = blockIdx.y;
    const int I = c_tri_i[t], J = c_tri_j[t];
    const int AI = I / 3, ci = I % 3, AJ = J / 3, cj = J % 3;
    for (int64_t E = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; E < mc; E += int64_t(gridDim.x) * blockDim.x) {
        const int ex = int(E % nxc);
        const int ey = int((E / nxc) % nyc);
        const int ez = int(E / (int64_t(nxc) * nyc));
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) {
            const int64_t e = (2 * ex + (c & 1)) + int64_t(nxf) * ((2 * ey + ((c >> 1) & 1)) + int64_t(nyf) * (2 * ez + (c >> 2)));
            for (int a = 0; a < 8; ++a) {
                const double wa = pc_weight(c, a, AI);
                if (wa == 0.0) continue;
                const int r = 3 * a + ci;
                for (int b = 0; b < 8; ++b) {
                    const double wb = pc_weight(c, b, AJ);
                    if (wb == 0.0) continue;
                    const int s = 3 * b + cj;
                    const int tt = r <= s ? tri_index(r, s) : tri_index(s, r);
                    acc += wa * wb * Af[tt * mf + e];
                }
            }
        }
        Ac[t * mc + E] = acc;
    }
}

void launch_build_coarser(pbm_grid* g, int k, cudaStream_t st) {
    const Geom& F = g->L[k].g;
    const int64_t mc = g->L[k + 1].g.m();
    dim3 grid(unsigned(std::max<int64_t>(1, std::min<int64_t>((mc + 127) / 128, 64))), NTRI);
    k_build_coarser<<<grid, 128, 0, st>>>(F.nx, F.ny, F.nz, g->L[k].A64, g->L[k + 1].A64);
    PBM_LAUNCH("build coarser");
}

void launch_coarse_to_f32(pbm_grid* g, int k, cudaStream_t st) {
    Level& L = g->L[k];
    if (L.A32) launch_cast(L.A64, false, L.A32, true, int64_t(NTRI) * L.g.m(), st);
    if (L.bord32) launch_cast(L.bord64, false, L.bord32, true, L.g.n(), st);
}

void upload_tri_tables() {
    static bool done = false;
    if (done) return;
    int ti[NTRI], tj[NTRI];
    for (int i = 0; i < 24; ++i)
        for (int j = i; j < 24; ++j) {
            ti[tri_index(i, j)] = i;
            tj[tri_index(i, j)] = j;
        }
    PBM_CUDA(cudaMemcpyToSymbol(c_tri_i, ti, sizeof(ti)));
    PBM_CUDA(cudaMemcpyToSymbol(c_tri_j, tj, sizeof(tj)));
    done = true;
}

// ------------------------------------------------------------------------------------------------
// coarsest level: dense assembly, Cholesky, explicit inverse (one CTA)
// ------------------------------------------------------------------------------------------------
__global__ void k_coarsest_factor(int nx, int ny, int nz, int support, const double* __restrict__ A,
                                  const double* __restrict__ bord, double s_alpha, int op_s, double* __restrict__ M,
                                  double* __restrict__ Inv, int* flag) {
    const int64_t m = int64_t(nx) * ny * nz;
    const int n = 3 * (nx + 1) * (ny + 1) * (nz + 1);
    const int N = n + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
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
    // Cholesky (lower, in place)
    __shared__ double piv;
    for (int j = 0; j < N; ++j) {
        if (tid == 0) {
            const double a = M[j * N + j];
            if (!(a > 0.0)) *flag = 1;
            piv = a > 0.0 ? sqrt(a) : 1.0;
            M[j * N + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < N; i += nt) M[i * N + j] /= piv;
        __syncthreads();
        const int rem = N - j - 1;
        for (int t = tid; t < rem * rem; t += nt) {
            const int i = j + 1 + t / rem, k = j + 1 + t % rem;
            if (k <= i) M[i * N + k] -= M[i * N + j] * M[k * N + j];
        }
        __syncthreads();
    }
    // Inv := L^{-1} (column by column, forward substitution), stored in the upper part of Inv rows
    for (int col = tid; col < N; col += nt) {
        for (int i = 0; i < N; ++i) {
            double s = (i == col) ? 1.0 : 0.0;
            for (int k = col; k < i; ++k) s -= M[i * N + k] * Inv[k * N + col];
            Inv[i * N + col] = (i < col) ? 0.0 : s / M[i * N + i];
        }
    }
    __syncthreads();
    // A^{-1} = L^{-T} L^{-1}: entry (r, c) = sum_k Linv[k][r] Linv[k][c], k >= max(r, c); store in M
    for (int t = tid; t < N * N; t += nt) {
        const int r = t / N, c = t % N;
        double s = 0.0;
        for (int k = (r > c ? r : c); k < N; ++k) s += Inv[k * N + r] * Inv[k * N + c];
        M[t] = s;
    }
    __syncthreads();
    for (int t = tid; t < N * N; t += nt) Inv[t] = M[t];
}

void build_coarsest(pbm_grid* g, bool op_s, cudaStream_t st) {
    const int kc = g->levels - 1;
    Level& L = g->L[kc];
    PBM_CUDA(cudaMemsetAsync(&g->sc->flags[0], 0, sizeof(int), st));
    if (kc == 0) fail(PBM_EINVAL, "a single-level hierarchy has no coarse operator (use levels >= 2)");
    k_coarsest_factor<<<1, 512, 0, st>>>(L.g.nx, L.g.ny, L.g.nz, L.g.support, L.A64, L.bord64, g->s_alpha, op_s ? 1 : 0,
                                         g->cwork, g->cinv, &g->sc->flags[0]);
    PBM_LAUNCH("coarsest factor");
}

// x = Inv b on the coarsest level (warp per row, FP64 accumulation)
template <class T>
__global__ void k_coarsest_solve(int N, int n_vec, const double* __restrict__ Inv, const T* __restrict__ b,
                                 T* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n_vec) return;
    double s = 0.0;
    for (int c = lane; c < n_vec; c += 32) s += Inv[row * N + c] * double(b[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = T(s);
}

void launch_coarsest_solve(pbm_grid* g, bool fp32, const void* b, void* x, bool with_alpha, cudaStream_t st) {
    const int N = g->nc + 1;
    const int nv = with_alpha ? N : N - 1;
    const int blocks = (nv * 32 + 255) / 256;
    if (fp32) k_coarsest_solve<float><<<blocks, 256, 0, st>>>(N, nv, g->cinv, (const float*)b, (float*)x);
    else k_coarsest_solve<double><<<blocks, 256, 0, st>>>(N, nv, g->cinv, (const double*)b, (double*)x);
    PBM_LAUNCH("coarsest solve");
}

}  // namespace pbm
