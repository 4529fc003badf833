// Single-pass FP32 fine-level operator: K(w) x and the S operator of eq. (S), with the fused apply /
// residual / damped-Jacobi epilogues (Section 5.1) and the Krylov dot products.
//
// In FP32 the operator is bound by memory traffic, not by arithmetic, so this kernel trades a little
// recomputation for traffic: every CTA owns a TX x TY tile of node columns and marches up a chunk of
// DZ node planes. It computes the (TX + 1) x (TY + 1) element columns around its tile, so the
// elements on tile borders are computed by two CTAs (and the element layer below a chunk by two
// chunks), and nothing but the inputs and the output goes through global memory:
//   * the node plane above the current element layer (x, and u for S) is staged in shared memory
//     with a one-node halo; the global loads of the plane after it are issued before the element
//     arithmetic of the current layer (software prefetch into registers);
//   * one thread per element column applies K_e = H^T Khat H (the factored element matrix, see
//     pbm_internal.h): the xy part of the transform of each plane is shared by the two layers that
//     touch it, and the top face of every element stays in registers until the next layer adds its
//     bottom face;
//   * the four element columns around a node exchange their corner values through shared memory;
//     the thread that owns the node sums them in a fixed order and applies the epilogue.
// The alpha row of S counts every element once (in the CTA and chunk that own its upper corner
// node). Per-CTA partial sums of the dot product and of the alpha row are finished by the last CTA
// in a fixed order, so results are bit-reproducible for a given tile plan.
#include <algorithm>

#include "fp32_elem.h"
#include "pbm_internal.h"

namespace pbm {

constexpr int FSLOT = 4;   // staging slots per thread: 3 (TX + 2)(TY + 2) <= FSLOT * NT

struct FusedArgs {
    int nx, ny, nz, support;
    int TX, TY, DZ, gx, gy;
    int64_t n;
    const float* x;
    const float* u;       // displacement (S)
    const float* w;       // element weights
    const float* d;       // Schur weights (S)
    float* y;
    const float* b;
    const float* idiag;
    const double* omega;
    int mode, with_alpha, dot_slot;
    KeHat2 K;
    double* partials;     // 2 * gridDim.x
    DevScalars* sc;
    unsigned int* counter;   // last-CTA counter
};

// transformed xy quad of the element column at staged coordinates (lx, ly) of a staged plane (nodes
// as float4, supported nodes already zero), components (x, y) paired
__device__ __forceinline__ void fused_quad2(const float4* __restrict__ s, int NW, int lx, int ly, float2 (&Q01)[4],
                                            float (&Q2)[4]) {
    float2 v01[4];
    float v2[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float4 p = s[(ly + (a >> 1)) * NW + lx + (a & 1)];
        v01[a] = make_float2(p.x, p.y);
        v2[a] = p.z;
    }
    const float2 s0 = add2(v01[0], v01[1]), d0 = sub2(v01[1], v01[0]);
    const float2 s1 = add2(v01[2], v01[3]), d1 = sub2(v01[3], v01[2]);
    Q01[0] = add2(s0, s1);
    Q01[1] = add2(d0, d1);
    Q01[2] = sub2(s1, s0);
    Q01[3] = sub2(d1, d0);
    const float t0 = v2[0] + v2[1], e0 = v2[1] - v2[0];
    const float t1 = v2[2] + v2[3], e1 = v2[3] - v2[2];
    Q2[0] = t0 + t1;
    Q2[1] = e0 + e1;
    Q2[2] = t1 - t0;
    Q2[3] = e1 - e0;
}

// MODE 0: K(w) x. MODE 2: S x with W_e = Khat H u_e recomputed from the staged u. NT threads per
// CTA, MINB resident CTAs per SM requested from the register allocator, an owner tile of TX x TY
// node columns (compile-time, so that every shared-memory offset is a constant).
template <int MODE, int NT, int MINB, int TX, int TY>
__global__ void __launch_bounds__(NT, MINB) k_fused_f32(FusedArgs P) {
    pdl_wait();
    constexpr bool S = MODE == 2;
    constexpr int EX = TX + 1, EY = TY + 1;
    constexpr int NW = TX + 2;             // staged nodes per row
    constexpr int SN = NW * (TY + 2);      // staged nodes per plane (float4 each, w unused)
    constexpr int RW = 3 * NW;             // floats per row of the global plane
    constexpr int SF = RW * (TY + 2);      // floats staged per plane
    constexpr int EC = EX * EY;
    static_assert(EC <= NT && TX * TY <= NT && SF <= FSLOT * NT, "tile does not fit the CTA");
    __shared__ float4 sx[2][SN];           // 2 planes of x
    __shared__ float4 su[S ? 2 : 1][S ? SN : 1];   // 2 planes of u (S)
    __shared__ float4 sq[4][EC];           // corner values of the element columns
    __shared__ double sred[NT / 32];
    __shared__ bool s_last;

    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny, nz = P.nz, support = P.support;
    const int bx = int(blockIdx.x % unsigned(P.gx));
    const int rest = int(blockIdx.x / unsigned(P.gx));
    const int by = rest % P.gy, bz = rest / P.gy;
    const int X0 = bx * TX, Y0 = by * TY;
    const int kz0 = bz * P.DZ, kz1 = min(kz0 + P.DZ, nz + 1);
    const int64_t plane = 3 * int64_t(nx + 1) * (ny + 1);

    // staging slots: float f = t + s NT of the staged plane (row f / RW, float f % RW of the row),
    // its offset in the global plane, its place in shared memory and the support bits of its node
    int gofs[FSLOT], sidx[FSLOT];
    int fbits = 0;
#pragma unroll
    for (int s = 0; s < FSLOT; ++s) {
        const int f = t + s * NT;
        gofs[s] = -2;
        sidx[s] = 0;
        if (f < SF) {
            const int row = f / RW, o = f - row * RW;
            const int lxn = o / 3, c = o - 3 * lxn;
            const int gxn = X0 - 1 + lxn, gyn = Y0 - 1 + row;
            const bool in = gxn >= 0 && gxn <= nx && gyn >= 0 && gyn <= ny;
            gofs[s] = in ? 3 * (gxn + (nx + 1) * gyn) + c : -1;
            sidx[s] = 4 * (row * NW + lxn) + c;
            if (in) fbits |= fixed_bits(support, nx, ny, nz, gxn, gyn) << (2 * s);
        }
    }
    float px[FSLOT], pu[FSLOT];
    auto fetch = [&](int k) {
        const float* xs = P.x + int64_t(k) * plane;
        const float* us = S ? P.u + int64_t(k) * plane : nullptr;
#pragma unroll
        for (int s = 0; s < FSLOT; ++s) {
            px[s] = gofs[s] >= 0 ? __ldg(xs + gofs[s]) : 0.0f;
            if (S) pu[s] = gofs[s] >= 0 ? __ldg(us + gofs[s]) : 0.0f;
        }
    };
    // writes the fetched plane into buffer `buf`, supported nodes zero (the masked vectors the element
    // matrices act on); first: the plane is plane 0
    auto stage = [&](int buf, bool first) {
        float* dx = reinterpret_cast<float*>(sx[buf]);
        float* du = reinterpret_cast<float*>(su[S ? buf : 0]);
        const int sh = first ? 1 : 0;
#pragma unroll
        for (int s = 0; s < FSLOT; ++s)
            if (gofs[s] != -2) {
                const bool fx = (fbits >> (2 * s + sh)) & 1;
                dx[sidx[s]] = fx ? 0.0f : px[s];
                if (S) du[sidx[s]] = fx ? 0.0f : pu[s];
            }
    };

    // element-column role
    const int lx = t % EX, ly = t / EX;
    const int ex = X0 - 1 + lx, ey = Y0 - 1 + ly;
    const bool ecol = t < EC && ex >= 0 && ex < nx && ey >= 0 && ey < ny;
    const bool designated = ecol && lx < TX && ly < TY;
    // owner role
    const int ox = t % TX, oy = t / TX;
    const int I = X0 + ox, J = Y0 + oy;
    const bool owner = t < TX * TY && I <= nx && J <= ny;
    const int obits = owner ? fixed_bits(support, nx, ny, nz, I, J) : 0;
    const int ooff = (oy + 1) * NW + ox + 1;   // staged node of the owner

    const float xa = S ? P.x[P.n] : 0.0f;
    // epilogue weights, converted once and only in their mode (no FP64 work in the other modes)
    float omF = 0.0f, c0F = 0.0f, c1F = 0.0f, c2F = 0.0f;
    bool c1nz = false;
    if (P.mode == EPI_JACOBI) omF = float(*P.omega);
    if (P.mode == EPI_CHEB) {
        c0F = float(P.omega[0]);
        c1F = float(P.omega[1]);
        c2F = float(P.omega[2]);
        c1nz = c1F != 0.0f;
    }
    const bool want_dot = P.dot_slot >= 0;
    float pdT = 0.0f, paT = 0.0f;

    const int kstart = max(kz0 - 1, 0);
    // per element column: xy-transformed quads of the plane below (x, and u for S) and the top face of the
    // previous layer, components (x, y) paired and z alone
    float2 Qlo01[4], Ulo01[4], carry01[4];
    float Qlo2[4], Ulo2[4], carry2[4];
    // element weights of the current layer, loaded one layer ahead
    const int64_t elayer = int64_t(nx) * ny;
    const float* wp = P.w + (ex + int64_t(nx) * (ey + int64_t(ny) * kstart));
    const float* dp = S ? P.d + (ex + int64_t(nx) * (ey + int64_t(ny) * kstart)) : nullptr;
    float wn = 0.0f, dn = 0.0f;
    if (ecol && kstart < nz) {
        wn = __ldg(wp);
        if (S) dn = __ldg(dp);
    }
    // the owner's dofs on plane k
    int64_t d0 = 3 * (I + int64_t(nx + 1) * (J + int64_t(ny + 1) * kz0));
    int cur = 0;                           // buffer of the plane below the current layer
    fetch(kstart);
    stage(cur, kstart == 0);
    if (kstart + 1 <= nz) fetch(kstart + 1);
    __syncthreads();
    if (ecol) {
        fused_quad2(sx[cur], NW, lx, ly, Qlo01, Qlo2);
        if (S) fused_quad2(su[S ? cur : 0], NW, lx, ly, Ulo01, Ulo2);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        carry01[q] = make_float2(0.0f, 0.0f);
        carry2[q] = 0.0f;
    }

    for (int k = kstart; k < kz1; ++k) {
        const bool layer = k < nz;
        const int nxt = cur ^ 1;           // buffer of plane k + 1
        if (layer) stage(nxt, false);
        __syncthreads();  // (a) plane k + 1 staged
        if (layer && k + 2 <= nz && k + 1 < kz1) fetch(k + 2);
        const float we = wn, de = dn;
        if (ecol && k + 1 < nz && k + 1 < kz1) {
            wp += elayer;
            wn = __ldg(wp);
            if (S) {
                dp += elayer;
                dn = __ldg(dp);
            }
        }
        // the owner's own x on plane k: staged (masked) unless the node is supported
        float4 xo4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const bool ofixed = (obits >> (k == 0 ? 1 : 0)) & 1;
        if (owner && k >= kz0) {
            if (ofixed) xo4 = make_float4(__ldg(P.x + d0), __ldg(P.x + d0 + 1), __ldg(P.x + d0 + 2), 0.0f);
            else xo4 = sx[cur][ooff];
        }
        float2 Bq01[4];
        float Bq2[4];
        if (ecol && layer) {
            float2 Qhi01[4];
            float Qhi2[4];
            fused_quad2(sx[nxt], NW, lx, ly, Qhi01, Qhi2);
            float2 X01[8], Y01[8];
            float X2[8], Y2[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                X01[q] = add2(Qlo01[q], Qhi01[q]);
                X01[q + 4] = sub2(Qhi01[q], Qlo01[q]);
                X2[q] = Qlo2[q] + Qhi2[q];
                X2[q + 4] = Qhi2[q] - Qlo2[q];
                Qlo01[q] = Qhi01[q];
                Qlo2[q] = Qhi2[q];
            }
            if (S) {
                float2 Uhi01[4], U01[8], W01[8];
                float Uhi2[4], U2[8], W2[8];
                fused_quad2(su[S ? nxt : 0], NW, lx, ly, Uhi01, Uhi2);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    U01[q] = add2(Ulo01[q], Uhi01[q]);
                    U01[q + 4] = sub2(Uhi01[q], Ulo01[q]);
                    U2[q] = Ulo2[q] + Uhi2[q];
                    U2[q + 4] = Uhi2[q] - Ulo2[q];
                    Ulo01[q] = Uhi01[q];
                    Ulo2[q] = Uhi2[q];
                }
                khat_apply2(P.K, U01, U2, W01, W2);
                float2 dot01 = make_float2(0.0f, 0.0f);
                float dot2 = 0.0f;
#pragma unroll
                for (int q = 1; q < 8; ++q) {
                    dot01 = fma2(W01[q], X01[q], dot01);
                    dot2 = fmaf(W2[q], X2[q], dot2);
                }
                const float te = de * ((dot01.x + dot01.y + dot2) - xa);
                if (designated && k + 1 >= kz0 && k + 1 < kz1) paT -= te;   // counted where its top plane is owned
                khat_apply2(P.K, X01, X2, Y01, Y2);
                const float2 we2 = make_float2(we, we), te2 = make_float2(te, te);
#pragma unroll
                for (int q = 1; q < 8; ++q) {
                    Y01[q] = fma2(te2, W01[q], mul2(we2, Y01[q]));
                    Y2[q] = fmaf(te, W2[q], we * Y2[q]);
                }
            } else {
                khat_apply2(P.K, X01, X2, Y01, Y2);
                const float2 we2 = make_float2(we, we);
#pragma unroll
                for (int q = 1; q < 8; ++q) {
                    Y01[q] = mul2(we2, Y01[q]);
                    Y2[q] *= we;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Bq01[q] = add2(carry01[q], sub2(Y01[q], Y01[q + 4]));
                carry01[q] = add2(Y01[q], Y01[q + 4]);
                Bq2[q] = carry2[q] + (Y2[q] - Y2[q + 4]);
                carry2[q] = Y2[q] + Y2[q + 4];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Bq01[q] = carry01[q];
                Bq2[q] = carry2[q];
                carry01[q] = make_float2(0.0f, 0.0f);
                carry2[q] = 0.0f;
            }
        }
        cur = nxt;
        if (k < kz0) continue;  // the layer below the chunk: only its top face is kept
        // inverse xy transform: the element column's values at its 4 corners of plane k
        if (t < EC) {
            const float2 a0 = sub2(Bq01[0], Bq01[1]), a1 = add2(Bq01[0], Bq01[1]);
            const float2 a2 = sub2(Bq01[2], Bq01[3]), a3 = add2(Bq01[2], Bq01[3]);
            const float b0 = Bq2[0] - Bq2[1], b1 = Bq2[0] + Bq2[1];
            const float b2 = Bq2[2] - Bq2[3], b3 = Bq2[2] + Bq2[3];
            const float2 o0 = sub2(a0, a2), o1 = sub2(a1, a3), o2 = add2(a0, a2), o3 = add2(a1, a3);
            sq[0][t] = make_float4(o0.x, o0.y, b0 - b2, 0.0f);
            sq[1][t] = make_float4(o1.x, o1.y, b1 - b3, 0.0f);
            sq[2][t] = make_float4(o2.x, o2.y, b0 + b2, 0.0f);
            sq[3][t] = make_float4(o3.x, o3.y, b1 + b3, 0.0f);
        }
        __syncthreads();  // (b) corner values of plane k complete
        if (owner) {
            const int gs_c = P.mode - EPI_GS0 - 3 * node_colour(I, J, k);   // Gauss-Seidel: the component updated
            float2 s01 = make_float2(0.0f, 0.0f);
            float s2 = 0.0f;
#pragma unroll
            for (int dj = 1; dj >= 0; --dj)
#pragma unroll
                for (int di = 1; di >= 0; --di) {
                    // element column (ox + 1 - di, oy + 1 - dj); the node is its corner (di, dj)
                    const float4 v = sq[di + 2 * dj][(oy + 1 - dj) * EX + (ox + 1 - di)];
                    s01 = add2(s01, make_float2(v.x, v.y));
                    s2 += v.z;
                }
            float s[3] = {s01.x, s01.y, s2};
            const float xo[3] = {xo4.x, xo4.y, xo4.z};
            if (ofixed) {
                s[0] = xo[0];
                s[1] = xo[1];
                s[2] = xo[2];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float o;
                if (P.mode == EPI_APPLY) {
                    o = s[c];
                    if (want_dot) pdT += o * xo[c];
                } else if (P.mode == EPI_RESID) {
                    o = __ldg(P.b + d0 + c) - s[c];
                    if (want_dot) pdT += o * o;
                } else if (P.mode == EPI_JACOBI) {
                    const float bb = __ldg(P.b + d0 + c);
                    o = xo[c] + omF * ((bb - s[c]) * __ldg(P.idiag + d0 + c));
                    if (want_dot) pdT += o * bb;
                } else if (P.mode == EPI_CHEB) {
                    const float bb = __ldg(P.b + d0 + c);
                    o = c0F * xo[c] + c2F * ((bb - s[c]) * __ldg(P.idiag + d0 + c));
                    if (c1nz) o -= c1F * P.y[d0 + c];
                    if (want_dot) pdT += o * bb;
                } else {
                    const float bb = __ldg(P.b + d0 + c);
                    o = gs_c == c ? xo[c] + (bb - s[c]) * __ldg(P.idiag + d0 + c) : xo[c];
                    if (want_dot) pdT += o * bb;
                }
                P.y[d0 + c] = o;
            }
        }
        d0 += plane;
    }

    // per-CTA partials; the last CTA finishes the dot and the alpha entry in a fixed order
    if (!want_dot && !P.with_alpha) return;
    const unsigned nblk = gridDim.x, blk = blockIdx.x;
    const double bd = fused_cta_sum<NT>(double(pdT), sred);
    const double ba = fused_cta_sum<NT>(double(paT), sred);
    if (t == 0) {
        P.partials[blk] = bd;
        P.partials[nblk + blk] = ba;
        __threadfence();
        s_last = atomicAdd(P.counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double td = 0.0, ta = 0.0;
    td = l2_strided_sum(P.partials, int(nblk), t, NT);
    ta = l2_strided_sum(P.partials + nblk, int(nblk), t, NT);
    double sd = fused_cta_sum<NT>(td, sred);
    const double sa = fused_cta_sum<NT>(ta, sred);
    if (t != 0) return;
    *P.counter = 0u;
    if (P.with_alpha) {
        const int64_t n = P.n;
        double o;
        if (P.mode == EPI_APPLY) {
            o = sa;
            sd += o * double(xa);
        } else if (P.mode == EPI_RESID) {
            o = double(P.b[n]) - sa;
            sd += o * o;
        } else if (P.mode == EPI_JACOBI) {
            const double bb = double(P.b[n]);
            o = double(xa) + *P.omega * ((bb - sa) * double(P.idiag[n]));
            sd += o * bb;
        } else if (P.mode == EPI_CHEB) {
            const double bb = double(P.b[n]);
            o = P.omega[0] * double(xa) + P.omega[2] * ((bb - sa) * double(P.idiag[n]));
            if (P.omega[1] != 0.0) o -= P.omega[1] * double(P.y[n]);
            sd += o * bb;
        } else {
            const double bb = double(P.b[n]);
            o = P.mode == EPI_GS0 + kGsColours ? double(xa) + (bb - sa) * double(P.idiag[n]) : double(xa);
            sd += o * bb;
        }
        P.y[n] = float(o);
    }
    if (want_dot) P.sc->red[P.dot_slot] = sd;
}

// ------------------------------------------------------------------------------------------------
// FP32 coarse levels: the same marching tile, with the stored Galerkin element matrices
// ------------------------------------------------------------------------------------------------
// Four threads per element column, one per xy corner q of the element: thread q forms the rows of
// local node q (bottom face, plane k) and of local node q + 4 (top face, plane k + 1), 144 FMAs per
// layer, reading the upper triangle (entry-major, A[t m + e]) of the 24 x 24 matrix. Its top rows
// are its carry into the next layer's bottom rows (the same xy corner). The coarse S adds the alpha
// border: y_u += b x_alpha, y_alpha = b . x + S_aa x_alpha.
struct CoarseArgs {
    int nx, ny, nz, support;
    int TX, TY, DZ, gx, gy;
    int64_t n, m;
    const float* A;
    const float* x;
    float* y;
    const float* b;
    const float* idiag;
    const double* omega;
    const float* bord;       // alpha border (S) or nullptr
    const double* s_alpha;   // S_alpha,alpha (S)
    int mode, with_alpha, dot_slot;
    double* partials;
    DevScalars* sc;
    unsigned int* counter;
};

constexpr int CSLOT = 2;   // staging slots per thread: 3 (TX + 2)(TY + 2) <= CSLOT * NT

template <int Q>
__device__ __forceinline__ void coarse_rows6(const float* __restrict__ Ae, int64_t m, const float (&xe)[24],
                                             float (&yb)[3], float (&yt)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int rb = 3 * Q + c, rt = 3 * (Q + 4) + c;
        float ab = 0.0f, at = 0.0f;
#pragma unroll
        for (int s = 0; s < 24; ++s) {
            const int tb = rb <= s ? tri_index(rb, s) : tri_index(s, rb);
            const int tt = rt <= s ? tri_index(rt, s) : tri_index(s, rt);
            ab = fmaf(__ldg(Ae + int64_t(tb) * m), xe[s], ab);
            at = fmaf(__ldg(Ae + int64_t(tt) * m), xe[s], at);
        }
        yb[c] = ab;
        yt[c] = at;
    }
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_fused_coarse_f32(CoarseArgs P) {
    pdl_wait();
    pdl_launch_if_small();
    extern __shared__ float4 fused_smem4[];
    __shared__ double sred[NT / 32];
    __shared__ bool s_last;

    const int TX = P.TX, TY = P.TY, EX = TX + 1, EY = TY + 1;
    const int NW = TX + 2;
    const int SN = NW * (TY + 2);
    const int RW = 3 * NW;
    const int SF = RW * (TY + 2);
    const int EC = EX * EY;
    float4* sx = fused_smem4;
    float4* sq = fused_smem4 + 2 * SN;

    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny, nz = P.nz, support = P.support;
    const int bx = int(blockIdx.x % unsigned(P.gx));
    const int rest = int(blockIdx.x / unsigned(P.gx));
    const int by = rest % P.gy, bz = rest / P.gy;
    const int X0 = bx * TX, Y0 = by * TY;
    const int kz0 = bz * P.DZ, kz1 = min(kz0 + P.DZ, nz + 1);
    const int64_t plane = 3 * int64_t(nx + 1) * (ny + 1);

    int gofs[CSLOT], sidx[CSLOT];
    int fbits = 0;
#pragma unroll
    for (int s = 0; s < CSLOT; ++s) {
        const int f = t + s * NT;
        gofs[s] = -2;
        sidx[s] = 0;
        if (f < SF) {
            const int row = f / RW, o = f - row * RW;
            const int lxn = o / 3, c = o - 3 * lxn;
            const int gxn = X0 - 1 + lxn, gyn = Y0 - 1 + row;
            const bool in = gxn >= 0 && gxn <= nx && gyn >= 0 && gyn <= ny;
            gofs[s] = in ? 3 * (gxn + (nx + 1) * gyn) + c : -1;
            sidx[s] = 4 * (row * NW + lxn) + c;
            if (in) fbits |= fixed_bits(support, nx, ny, nz, gxn, gyn) << (2 * s);
        }
    }
    float px[CSLOT];
    auto fetch = [&](int k) {
        const float* xs = P.x + int64_t(k) * plane;
#pragma unroll
        for (int s = 0; s < CSLOT; ++s) px[s] = gofs[s] >= 0 ? __ldg(xs + gofs[s]) : 0.0f;
    };
    auto stage = [&](int k) {
        float* dx = reinterpret_cast<float*>(sx + (k & 1) * SN);
        const int sh = k == 0 ? 1 : 0;
#pragma unroll
        for (int s = 0; s < CSLOT; ++s)
            if (gofs[s] != -2) dx[sidx[s]] = ((fbits >> (2 * s + sh)) & 1) ? 0.0f : px[s];
    };

    // element-column role: corner q of element column col
    const int q = t / EC, col = t - q * EC;
    const int lx = col % EX, ly = col / EX;
    const int ex = X0 - 1 + lx, ey = Y0 - 1 + ly;
    const bool ecol = q < 4 && ex >= 0 && ex < nx && ey >= 0 && ey < ny;
    // owner role
    const int ox = t % TX, oy = t / TX;
    const int I = X0 + ox, J = Y0 + oy;
    const bool owner = t < TX * TY && I <= nx && J <= ny;
    const int obits = owner ? fixed_bits(support, nx, ny, nz, I, J) : 0;

    const float xa = P.with_alpha ? P.x[P.n] : 0.0f;
    // epilogue weights, converted once and only in their mode (no FP64 work in the other modes)
    float omF = 0.0f, c0F = 0.0f, c1F = 0.0f, c2F = 0.0f;
    bool c1nz = false;
    if (P.mode == EPI_JACOBI) omF = float(*P.omega);
    if (P.mode == EPI_CHEB) {
        c0F = float(P.omega[0]);
        c1F = float(P.omega[1]);
        c2F = float(P.omega[2]);
        c1nz = c1F != 0.0f;
    }
    const bool want_dot = P.dot_slot >= 0;
    float pdT = 0.0f, paT = 0.0f;

    const int kstart = max(kz0 - 1, 0);
    const int64_t elayer = int64_t(nx) * ny;
    const int64_t e0 = ex + int64_t(nx) * ey;
    float carry[3] = {0.0f, 0.0f, 0.0f};
    fetch(kstart);
    stage(kstart);
    if (kstart + 1 <= nz) fetch(kstart + 1);

    for (int k = kstart; k < kz1; ++k) {
        const bool layer = k < nz;
        if (layer) stage(k + 1);
        __syncthreads();  // (a) planes k and k + 1 staged
        if (layer && k + 2 <= nz && k + 1 < kz1) fetch(k + 2);
        float4 xo4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const bool ofixed = (obits >> (k == 0 ? 1 : 0)) & 1;
        const int64_t d0 = 3 * (I + int64_t(nx + 1) * (J + int64_t(ny + 1) * k));
        if (owner && k >= kz0) {
            if (ofixed) xo4 = make_float4(__ldg(P.x + d0), __ldg(P.x + d0 + 1), __ldg(P.x + d0 + 2), 0.0f);
            else xo4 = sx[(k & 1) * SN + (oy + 1) * NW + ox + 1];
        }
        float yb[3] = {0.0f, 0.0f, 0.0f}, yt[3] = {0.0f, 0.0f, 0.0f};
        if (ecol && layer) {
            float xe[24];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float4 v = sx[((k + (a >> 2)) & 1) * SN + (ly + ((a >> 1) & 1)) * NW + lx + (a & 1)];
                xe[3 * a] = v.x;
                xe[3 * a + 1] = v.y;
                xe[3 * a + 2] = v.z;
            }
            const float* Ae = P.A + e0 + int64_t(k) * elayer;
            switch (q) {
                case 0: coarse_rows6<0>(Ae, P.m, xe, yb, yt); break;
                case 1: coarse_rows6<1>(Ae, P.m, xe, yb, yt); break;
                case 2: coarse_rows6<2>(Ae, P.m, xe, yb, yt); break;
                default: coarse_rows6<3>(Ae, P.m, xe, yb, yt); break;
            }
        }
        float ob[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ob[c] = carry[c] + yb[c];
            carry[c] = yt[c];
        }
        if (k < kz0) continue;
        if (q < 4) sq[q * EC + col] = make_float4(ob[0], ob[1], ob[2], 0.0f);
        __syncthreads();  // (b) corner values of plane k complete
        if (owner) {
            const int gs_c = P.mode - EPI_GS0 - 3 * node_colour(I, J, k);   // Gauss-Seidel: the component updated
            float s3[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int dj = 1; dj >= 0; --dj)
#pragma unroll
                for (int di = 1; di >= 0; --di) {
                    const float4 v = sq[(di + 2 * dj) * EC + (oy + 1 - dj) * EX + (ox + 1 - di)];
                    s3[0] += v.x;
                    s3[1] += v.y;
                    s3[2] += v.z;
                }
            const float xo[3] = {xo4.x, xo4.y, xo4.z};
            if (P.bord) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float bc = __ldg(P.bord + d0 + c);
                    s3[c] += bc * xa;
                    paT += bc * xo[c];
                }
            }
            if (ofixed) {
                s3[0] = xo[0];
                s3[1] = xo[1];
                s3[2] = xo[2];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float o;
                if (P.mode == EPI_APPLY) {
                    o = s3[c];
                    if (want_dot) pdT += o * xo[c];
                } else if (P.mode == EPI_RESID) {
                    o = __ldg(P.b + d0 + c) - s3[c];
                    if (want_dot) pdT += o * o;
                } else if (P.mode == EPI_JACOBI) {
                    const float bb = __ldg(P.b + d0 + c);
                    o = xo[c] + omF * ((bb - s3[c]) * __ldg(P.idiag + d0 + c));
                    if (want_dot) pdT += o * bb;
                } else if (P.mode == EPI_CHEB) {
                    const float bb = __ldg(P.b + d0 + c);
                    o = c0F * xo[c] + c2F * ((bb - s3[c]) * __ldg(P.idiag + d0 + c));
                    if (c1nz) o -= c1F * P.y[d0 + c];
                    if (want_dot) pdT += o * bb;
                } else {
                    const float bb = __ldg(P.b + d0 + c);
                    o = gs_c == c ? xo[c] + (bb - s3[c]) * __ldg(P.idiag + d0 + c) : xo[c];
                    if (want_dot) pdT += o * bb;
                }
                P.y[d0 + c] = o;
            }
        }
    }

    if (!want_dot && !P.with_alpha) return;
    const unsigned nblk = gridDim.x, blk = blockIdx.x;
    const double bd = fused_cta_sum<NT>(double(pdT), sred);
    const double ba = fused_cta_sum<NT>(double(paT), sred);
    if (t == 0) {
        P.partials[blk] = bd;
        P.partials[nblk + blk] = ba;
        __threadfence();
        s_last = atomicAdd(P.counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double td = 0.0, ta = 0.0;
    td = l2_strided_sum(P.partials, int(nblk), t, NT);
    ta = l2_strided_sum(P.partials + nblk, int(nblk), t, NT);
    double sd = fused_cta_sum<NT>(td, sred);
    const double sa = fused_cta_sum<NT>(ta, sred);
    if (t != 0) return;
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
        P.y[n] = float(o);
    }
    if (want_dot) P.sc->red[P.dot_slot] = sd;
}

// ------------------------------------------------------------------------------------------------
// tile plans
// ------------------------------------------------------------------------------------------------
// Plans of the fine kernel: threads per CTA, resident CTAs per SM asked of the register allocator, and
// the owner tile TX x TY ((TX + 1)(TY + 1) element columns fit the CTA; the staged plane,
// 3 (TX + 2)(TY + 2) floats, fits its staging slots). The list keeps the shapes that timed best on
// the grids of the workloads.
#define PBM_FUSED_PLANS(X)                                                                                  \
    X(0, 256, 2, 31, 7) X(1, 256, 2, 21, 10) X(2, 256, 2, 26, 8) X(3, 256, 2, 15, 15) X(4, 256, 1, 31, 7)    \
    X(5, 256, 1, 21, 10) X(6, 128, 4, 15, 7) X(7, 128, 4, 20, 5) X(8, 128, 4, 7, 15) X(9, 128, 4, 24, 4)     \
    X(10, 128, 3, 15, 7) X(11, 128, 3, 24, 4)
#define PBM_PLAN_ROW(i, nt, minb, tx, ty) {nt, minb, tx, ty},
static const int kFusedPlans[][4] = {PBM_FUSED_PLANS(PBM_PLAN_ROW)};
#undef PBM_PLAN_ROW
constexpr int kFusedNumPlans = int(sizeof(kFusedPlans) / sizeof(kFusedPlans[0]));

// Plan numbers: 0 .. kFusedNumPlans - 1 this file's tiles, kFusedNumPlans the tensor-core kernel (tc.cu), then
// the lane-strip kernel's plans (strip.cu).
static bool is_strip(int cand) { return cand > kFusedNumPlans; }

FusedPlan fused_plan(const Geom& G, int cand, bool op_s) {
    if (cand == kFusedNumPlans) {
        FusedPlan p = tc_plan(G, op_s);
        p.var = cand;
        return p;
    }
    if (is_strip(cand)) {
        FusedPlan p = strip_plan(G, cand - kFusedNumPlans - 1);
        p.var = cand;
        return p;
    }
    FusedPlan p{};
    p.var = cand;
    const int per_sm = kFusedPlans[cand][1];
    p.TX = kFusedPlans[cand][2];
    p.TY = kFusedPlans[cand][3];
    p.gx = (G.nx + 1 + p.TX - 1) / p.TX;
    p.gy = (G.ny + 1 + p.TY - 1) / p.TY;
    const int planes = G.nz + 1;
    const int tiles = p.gx * p.gy;
    const int sms = num_sms();
    // chunk length: with per_sm resident CTAs per SM a launch takes about waves x (DZ + 1) plane
    // steps; take the shortest, then the fewest CTAs
    double best = 1e300;
    p.DZ = planes;
    for (int dz = std::max(1, std::min(planes, 2)); dz <= planes; ++dz) {
        const int gz = (planes + dz - 1) / dz;
        if (dz > 1 && (planes + dz - 2) / (dz - 1) == gz && dz != planes) continue;  // same split, shorter dz
        const double waves = double((int64_t(tiles) * gz + sms * per_sm - 1) / (sms * per_sm));
        const double cost = waves * (dz + 1);
        if (cost < best - 1e-9) {
            best = cost;
            p.DZ = dz;
        }
    }
    p.gz = (planes + p.DZ - 1) / p.DZ;
    return p;
}

int fused_num_plans() { return kFusedNumPlans + 1 + strip_num_plans(); }

int fused_tc_plan() { return kFusedNumPlans; }

int fused_blocks(const FusedPlan& p) { return p.gx * p.gy * p.gz; }

int fused_threads(const FusedPlan& p) {
    if (is_strip(p.var)) return strip_threads(p.var - kFusedNumPlans - 1);
    return p.var == kFusedNumPlans ? 256 : kFusedPlans[p.var][0];
}

// plan used until the autotuner has timed the candidates (and for grids it does not tune): fewest
// plane steps per SM (waves x (DZ + 1) / resident CTAs), then fewest element columns computed
int fused_default_plan(const Geom& G) {
    int best = 0;
    double bc = 1e300;
    const int sms = num_sms();
    for (int c = 0; c < kFusedNumPlans; ++c) {
        const FusedPlan p = fused_plan(G, c);
        const int per_sm = kFusedPlans[p.var][1];
        const int blocks = fused_blocks(p);
        const double waves = double((blocks + sms * per_sm - 1) / (sms * per_sm));
        const double cols = double(p.gx) * (p.TX + 1) * p.gy * (p.TY + 1);
        const double cost = waves * (p.DZ + 1) / per_sm * 1e9 + cols * (p.DZ + 1) / p.DZ;
        if (cost < bc) {
            bc = cost;
            best = c;
        }
    }
    return best;
}

template <int MODE>
static void fused_launch(const FusedPlan& p, int blocks, const FusedArgs& P, cudaStream_t st) {
    switch (p.var) {
#define PBM_PLAN_CASE(i, nt, minb, tx, ty) \
    case i: launch_pdl(k_fused_f32<MODE, nt, minb, tx, ty>, dim3(blocks), dim3(nt), 0, st, P); break;
        PBM_FUSED_PLANS(PBM_PLAN_CASE)
#undef PBM_PLAN_CASE
        default: fail(PBM_EINVAL, "fused operator: unknown plan");
    }
}

void fused_fine_f32(const FusedPlan& p, const RedSet& r, const Geom& G, const KeHat& kh, const TcMatrix& tm,
                    const float* w, const float* d, const float* u, const ApplyArgs& a, cudaStream_t st) {
    if (p.var == kFusedNumPlans) {
        tc_fine_f32(p, r, G, tm, w, d, u, a, st);
        return;
    }
    if (is_strip(p.var)) {
        strip_fine_f32(p.var - kFusedNumPlans - 1, p, r, G, kh, w, d, u, a, st);
        return;
    }
    const bool s = d != nullptr;
    const int nt = fused_threads(p);
    if ((p.TX + 1) * (p.TY + 1) > nt || 3 * (p.TX + 2) * (p.TY + 2) > FSLOT * nt)
        fail(PBM_EINVAL, "fused operator: tile does not fit the CTA");
    const int blocks = fused_blocks(p);
    if (2 * int64_t(blocks) > r.len) fail(PBM_EINVAL, "grid too large for the partials buffer");
    FusedArgs P{};
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.support = G.support;
    P.TX = p.TX;
    P.TY = p.TY;
    P.DZ = p.DZ;
    P.gx = p.gx;
    P.gy = p.gy;
    P.n = G.n();
    P.x = (const float*)a.x;
    P.u = u;
    P.w = w;
    P.d = d;
    P.y = (float*)a.y;
    P.b = (const float*)a.b;
    P.idiag = (const float*)a.diag;
    P.omega = a.omega;
    P.mode = a.mode;
    P.with_alpha = (s && a.with_alpha) ? 1 : 0;
    P.dot_slot = a.dot_slot;
    for (int q = 0; q < 8; ++q) {
        P.K.dg01[q] = make_float2(float(kh.dg[0][q]), float(kh.dg[1][q]));
        P.K.dg2[q] = float(kh.dg[2][q]);
    }
    for (int b = 0; b < 2; ++b) {
        P.K.lam4[b] = float(kh.lam4[b]);
        P.K.mu4[b] = float(kh.mu4[b]);
    }
    P.partials = r.partials;
    P.sc = r.sc;
    P.counter = r.counter;
    if (s) fused_launch<2>(p, blocks, P, st);
    else fused_launch<0>(p, blocks, P, st);
    PBM_LAUNCH("fused FP32 fine operator");
}

// ---- coarse-level plans: CTA size, resident CTAs per SM, owner tile (4 (TX+1)(TY+1) = threads) ----
static const int kCoarsePlans[][4] = {{256, 2, 7, 7}, {256, 2, 15, 3}, {128, 4, 7, 3}, {128, 4, 3, 7},
                                      {256, 1, 7, 7}, {128, 2, 7, 3}};
constexpr int kCoarseNumPlans = int(sizeof(kCoarsePlans) / sizeof(kCoarsePlans[0]));

int fused_coarse_num_plans() { return kCoarseNumPlans; }

FusedPlan fused_coarse_plan(const Geom& G, int cand) {
    FusedPlan p{};
    p.var = cand;
    const int per_sm = kCoarsePlans[cand][1];
    p.TX = kCoarsePlans[cand][2];
    p.TY = kCoarsePlans[cand][3];
    p.gx = (G.nx + 1 + p.TX - 1) / p.TX;
    p.gy = (G.ny + 1 + p.TY - 1) / p.TY;
    const int planes = G.nz + 1;
    const int tiles = p.gx * p.gy;
    const int sms = num_sms();
    double best = 1e300;
    p.DZ = planes;
    for (int dz = std::max(1, std::min(planes, 2)); dz <= planes; ++dz) {
        const int gz = (planes + dz - 1) / dz;
        if (dz > 1 && (planes + dz - 2) / (dz - 1) == gz && dz != planes) continue;
        const double waves = double((int64_t(tiles) * gz + sms * per_sm - 1) / (sms * per_sm));
        const double cost = waves * (dz + 1);
        if (cost < best - 1e-9) {
            best = cost;
            p.DZ = dz;
        }
    }
    p.gz = (planes + p.DZ - 1) / p.DZ;
    return p;
}

void fused_coarse_f32(const FusedPlan& p, const RedSet& r, const Geom& G, const float* A, const float* bord,
                      const double* s_alpha, const ApplyArgs& a, cudaStream_t st) {
    const int nt = kCoarsePlans[p.var][0];
    if (4 * (p.TX + 1) * (p.TY + 1) != nt || 3 * (p.TX + 2) * (p.TY + 2) > CSLOT * nt || p.TX * p.TY > nt)
        fail(PBM_EINVAL, "fused coarse operator: tile does not fit the CTA");
    const int blocks = p.gx * p.gy * p.gz;
    if (2 * int64_t(blocks) > r.len) fail(PBM_EINVAL, "grid too large for the partials buffer");
    CoarseArgs P{};
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.support = G.support;
    P.TX = p.TX;
    P.TY = p.TY;
    P.DZ = p.DZ;
    P.gx = p.gx;
    P.gy = p.gy;
    P.n = G.n();
    P.m = G.m();
    P.A = A;
    P.x = (const float*)a.x;
    P.y = (float*)a.y;
    P.b = (const float*)a.b;
    P.idiag = (const float*)a.diag;
    P.omega = a.omega;
    P.bord = a.with_alpha ? bord : nullptr;
    P.s_alpha = s_alpha;
    P.mode = a.mode;
    P.with_alpha = a.with_alpha ? 1 : 0;
    P.dot_slot = a.dot_slot;
    P.partials = r.partials;
    P.sc = r.sc;
    P.counter = r.counter;
    const size_t smem = sizeof(float4) * (size_t(2 * (p.TX + 2) * (p.TY + 2)) + size_t(4 * (p.TX + 1) * (p.TY + 1)));
    switch (p.var) {
        case 0:
        case 1: launch_pdl(k_fused_coarse_f32<256, 2>, dim3(blocks), dim3(256), smem, st, P); break;
        case 2:
        case 3: launch_pdl(k_fused_coarse_f32<128, 4>, dim3(blocks), dim3(128), smem, st, P); break;
        case 4: launch_pdl(k_fused_coarse_f32<256, 1>, dim3(blocks), dim3(256), smem, st, P); break;
        default: launch_pdl(k_fused_coarse_f32<128, 2>, dim3(blocks), dim3(128), smem, st, P); break;
    }
    PBM_LAUNCH("fused FP32 coarse operator");
}

}  // namespace pbm
