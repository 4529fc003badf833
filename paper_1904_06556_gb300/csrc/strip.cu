// Single-pass FP32 fine-level operator in lane strips: K(w) x and the S operator of eq. (S) with the fused
// apply / residual / damped-Jacobi / Chebyshev / Gauss-Seidel epilogues (Section 5.1) and the Krylov dot
// products, organised so that almost every value an element shares with its neighbours stays in registers.
//
// A warp's 32 lanes are 32 consecutive node columns i = X0 - 1 + lane (consecutive lanes read consecutive
// nodes: every global access is coalesced). Lane l <= 30 owns the element column i, between its node column
// and the next lane's; each lane walks a strip of NYB element rows in y and the warp marches up the planes in
// z. The element matrix is applied in its factored form H^T Khat H (pbm_internal.h) with the transform split
// by direction and every partial result shared as far as it goes:
//   * x: the sum and difference of the two node columns of an element ("x-pairs") are formed once per node
//     row and plane, from the lane's own column and its right neighbour's (one shuffle per value), and used
//     by the two element rows and the two layers that touch them;
//   * y: the element's face quad (sum / difference of its two x-pairs) is formed per element and plane;
//   * z: the element's 24 transformed coefficients are the sum and difference of its two face quads.
// The output goes back the same way: each element's bottom and top faces are split into the x-pair form of
// their node rows and accumulated per row (the top faces are the carry into the next plane), and a node's
// value is its own column's part plus the part the lane on its left computed (one shuffle per value). The
// node row between two warps is completed through shared memory (one float4 per lane and plane, double
// buffered so that one barrier per plane suffices). Nothing but the inputs and the output goes through
// global memory, and no element value is recomputed except on the CTA's one-column and one-row halo and on
// the layer below each plane chunk.
//
// The alpha row of S counts every element once (in the CTA and chunk that own its upper corner node). Per-CTA
// partial sums of the dot product and of the alpha row are finished by the last CTA in a fixed order, so the
// results are bit-reproducible for a given plan.
#include <algorithm>

#include "fp32_elem.h"
#include "pbm_internal.h"

namespace pbm {

namespace {

constexpr int kStripOwnedX = 30;   // owned node columns per warp (lanes 1 .. 30)

// a 3-vector with components (x, y) paired for the packed instructions and z alone
struct V3 {
    float2 a;
    float b;
};
__device__ __forceinline__ V3 v3zero() { return V3{make_float2(0.0f, 0.0f), 0.0f}; }
__device__ __forceinline__ V3 operator+(V3 p, V3 q) { return V3{add2(p.a, q.a), p.b + q.b}; }
__device__ __forceinline__ V3 operator-(V3 p, V3 q) { return V3{sub2(p.a, q.a), p.b - q.b}; }

// the x-pair of a node row: s = v(i + 1) + v(i), d = v(i + 1) - v(i)
struct XP {
    V3 s, d;
};

struct StripArgs {
    int nx, ny, nz, support;
    int DZ, gx, gy;
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
    unsigned int* counter;
};

// face quad of element row r from the x-pairs of its two node rows (fused.cu's fused_quad2 convention:
// Q0 = sum, Q1 = x-difference, Q2 = y-difference, Q3 = both)
__device__ __forceinline__ void face_quad(const XP& lo, const XP& hi, V3 (&Q)[4]) {
    Q[0] = lo.s + hi.s;
    Q[1] = lo.d + hi.d;
    Q[2] = hi.s - lo.s;
    Q[3] = hi.d - lo.d;
}

// the 24 transformed coefficients of an element from the face quads of its bottom and top planes
__device__ __forceinline__ void element_coeffs(const V3 (&Qb)[4], const V3 (&Qt)[4], float2 (&X01)[8], float (&X2)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const V3 p = Qb[q] + Qt[q], m = Qt[q] - Qb[q];
        X01[q] = p.a;
        X2[q] = p.b;
        X01[q + 4] = m.a;
        X2[q + 4] = m.b;
    }
}

// adds a face F (transformed, 4 q-values) to the x-pair accumulators of its low and high node rows
__device__ __forceinline__ void face_to_rows(const V3 (&F)[4], XP& low, XP& high) {
    low.s = low.s + (F[0] - F[2]);
    low.d = low.d + (F[1] - F[3]);
    high.s = high.s + (F[0] + F[2]);
    high.d = high.d + (F[1] + F[3]);
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// node value of a row from its x-pair accumulator: the left part of the own column plus the right part the
// lane on the left computed (lane 0's value is incomplete; it is never owned)
__device__ __forceinline__ V3 row_total(const XP& a) {
    const V3 L = a.s - a.d, Rt = a.s + a.d;
    V3 Rp;
    Rp.a = make_float2(shfl_up1(Rt.a.x), shfl_up1(Rt.a.y));
    Rp.b = shfl_up1(Rt.b);
    return L + Rp;
}

}  // namespace

// MODE 0: K(w) x. MODE 2: S x with W_e = Khat H u_e recomputed from u. NW warps per CTA, NYB element rows per
// warp, MINB resident CTAs per SM asked of the register allocator.
template <int MODE, int NYB, int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) k_strip_f32(StripArgs P) {
    pdl_wait();
    constexpr bool S = MODE == 2;
    constexpr int NT = 32 * NW;
    constexpr int R = NW * NYB;            // element rows of the CTA
    __shared__ float4 sy[2][NW][32];       // node totals of each warp's top row, by plane parity
    __shared__ double sred[NW];
    __shared__ bool s_last;

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nx = P.nx, ny = P.ny, nz = P.nz, support = P.support;
    const int bx = int(blockIdx.x % unsigned(P.gx));
    const int rest = int(blockIdx.x / unsigned(P.gx));
    const int by = rest % P.gy, bz = rest / P.gy;
    const int X0 = bx * kStripOwnedX, Y0 = by * (R - 1);
    const int kz0 = bz * P.DZ, kz1 = min(kz0 + P.DZ, nz + 1);
    const int i = X0 - 1 + lane;           // node column (and element column) of this lane
    const int jb = Y0 - 1 + wid * NYB;     // first element row and node row of this warp
    const int64_t plane = 3 * int64_t(nx + 1) * (ny + 1);
    const int64_t elayer = int64_t(nx) * ny;

    // per node row r = 0 .. NYB: in range and not supported, for planes k >= 1 (bit r) and plane 0 (bit 16 + r)
    unsigned okm = 0, fixm = 0;
    int noff[NYB + 1];                     // node offsets (floats) within a plane
#pragma unroll
    for (int r = 0; r <= NYB; ++r) {
        const int j = jb + r;
        const bool in = i >= 0 && i <= nx && j >= 0 && j <= ny;
        noff[r] = in ? 3 * (i + (nx + 1) * j) : 0;
        if (in) {
            const int fb = fixed_bits(support, nx, ny, nz, i, j);
            if (!(fb & 1)) okm |= 1u << r;
            if (!(fb & 2)) okm |= 1u << (16 + r);
            fixm |= unsigned(fb & 1) << r;
            fixm |= unsigned((fb >> 1) & 1) << (16 + r);
        }
    }
    // element rows r = 0 .. NYB - 1 that exist (lanes 0 .. 30), and those whose alpha term this CTA counts
    unsigned em = 0, am = 0;
    int eoff[NYB];
#pragma unroll
    for (int r = 0; r < NYB; ++r) {
        const int j = jb + r;
        const bool e = lane <= 30 && i >= 0 && i < nx && j >= 0 && j < ny;
        eoff[r] = e ? i + nx * j : 0;
        if (e) em |= 1u << r;
        if (e && lane >= 1 && j >= Y0) am |= 1u << r;
    }

    const float xa = S ? P.x[P.n] : 0.0f;
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

    // raw node values of the lane's column (rows 0 .. NYB) of one plane, zero where not in range or supported
    float rx[NYB + 1][3], ru[S ? NYB + 1 : 1][3];
    auto fetch = [&](int k) {
        const unsigned ok = k == 0 ? (okm >> 16) : okm;
        const float* xs = P.x + int64_t(k) * plane;
        const float* us = S ? P.u + int64_t(k) * plane : nullptr;
#pragma unroll
        for (int r = 0; r <= NYB; ++r) {
            const bool v = (ok >> r) & 1u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rx[r][c] = v ? __ldg(xs + noff[r] + c) : 0.0f;
                if (S) ru[r][c] = v ? __ldg(us + noff[r] + c) : 0.0f;
            }
        }
    };
    // x-pairs of one node row from the lane's column and the right neighbour's
    auto xpair = [&](const float (&v)[3]) {
        const float r0 = shfl_dn1(v[0]), r1 = shfl_dn1(v[1]), r2 = shfl_dn1(v[2]);
        XP p;
        p.s = V3{make_float2(r0 + v[0], r1 + v[1]), r2 + v[2]};
        p.d = V3{make_float2(r0 - v[0], r1 - v[1]), r2 - v[2]};
        return p;
    };

    const int kstart = max(kz0 - 1, 0);
    XP xl[NYB + 1], ul[S ? NYB + 1 : 1];   // x-pairs of the plane below the current layer
    XP acc[NYB + 1];                       // x-pair accumulators of the current plane's node rows
    fetch(kstart);
#pragma unroll
    for (int r = 0; r <= NYB; ++r) {
        xl[r] = xpair(rx[r]);
        if (S) ul[r] = xpair(ru[r]);
        acc[r].s = acc[r].d = v3zero();
    }
    if (kstart + 1 <= nz) fetch(kstart + 1);
    float wn[NYB], dn[S ? NYB : 1];
    auto fetch_w = [&](int k) {
#pragma unroll
        for (int r = 0; r < NYB; ++r) {
            const bool e = (em >> r) & 1u;
            wn[r] = e ? __ldg(P.w + int64_t(k) * elayer + eoff[r]) : 0.0f;
            if (S) dn[r] = e ? __ldg(P.d + int64_t(k) * elayer + eoff[r]) : 0.0f;
        }
    };
    if (kstart < nz) fetch_w(kstart);

    for (int k = kstart; k < kz1; ++k) {
        const bool layer = k < nz;
        XP nxt[NYB + 1];                   // x-pair accumulators of plane k + 1 (the top faces)
#pragma unroll
        for (int r = 0; r <= NYB; ++r) nxt[r].s = nxt[r].d = v3zero();
        if (layer) {
            XP xh[NYB + 1], uh[S ? NYB + 1 : 1];
#pragma unroll
            for (int r = 0; r <= NYB; ++r) {
                xh[r] = xpair(rx[r]);
                if (S) uh[r] = xpair(ru[r]);
            }
            if (k + 2 <= nz && k + 1 < kz1) fetch(k + 2);
            float we[NYB], de[S ? NYB : 1];
#pragma unroll
            for (int r = 0; r < NYB; ++r) {
                we[r] = wn[r];
                if (S) de[r] = dn[r];
            }
            if (k + 1 < nz && k + 1 < kz1) fetch_w(k + 1);
            const bool count_alpha = k + 1 >= kz0 && k + 1 < kz1;
#pragma unroll
            for (int r = 0; r < NYB; ++r) {
                V3 Qb[4], Qt[4];
                face_quad(xl[r], xl[r + 1], Qb);
                face_quad(xh[r], xh[r + 1], Qt);
                float2 X01[8], Y01[8];
                float X2[8], Y2[8];
                element_coeffs(Qb, Qt, X01, X2);
                khat_apply2(P.K, X01, X2, Y01, Y2);
                const float2 we2 = make_float2(we[r], we[r]);
                if (S) {
                    V3 Ub[4], Ut[4];
                    face_quad(ul[r], ul[r + 1], Ub);
                    face_quad(uh[r], uh[r + 1], Ut);
                    float2 U01[8], W01[8];
                    float U2[8], W2[8];
                    element_coeffs(Ub, Ut, U01, U2);
                    khat_apply2(P.K, U01, U2, W01, W2);
                    float2 dot01 = make_float2(0.0f, 0.0f);
                    float dot2 = 0.0f;
#pragma unroll
                    for (int q = 1; q < 8; ++q) {
                        dot01 = fma2(W01[q], X01[q], dot01);
                        dot2 = fmaf(W2[q], X2[q], dot2);
                    }
                    const float te = de[r] * ((dot01.x + dot01.y + dot2) - xa);
                    if (count_alpha && ((am >> r) & 1u)) paT -= te;
                    const float2 te2 = make_float2(te, te);
#pragma unroll
                    for (int q = 1; q < 8; ++q) {
                        Y01[q] = fma2(te2, W01[q], mul2(we2, Y01[q]));
                        Y2[q] = fmaf(te, W2[q], we[r] * Y2[q]);
                    }
                } else {
#pragma unroll
                    for (int q = 1; q < 8; ++q) {
                        Y01[q] = mul2(we2, Y01[q]);
                        Y2[q] *= we[r];
                    }
                }
                V3 B[4], T[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const V3 lo = V3{Y01[q], Y2[q]}, hi = V3{Y01[q + 4], Y2[q + 4]};
                    B[q] = lo - hi;
                    T[q] = lo + hi;
                }
                face_to_rows(B, acc[r], acc[r + 1]);
                face_to_rows(T, nxt[r], nxt[r + 1]);
            }
#pragma unroll
            for (int r = 0; r <= NYB; ++r) {
                xl[r] = xh[r];
                if (S) ul[r] = uh[r];
            }
        }
        if (k >= kz0) {
            // node totals of plane k: rows 1 .. NYB - 1 complete in the warp, row NYB shared with the warp above,
            // row 0 with the warp below
            const int64_t pbase = int64_t(k) * plane;
            auto epilogue = [&](int r, V3 s) {
                const int j = jb + r;
                if (lane < 1 || lane > 30 || i > nx || j < 0 || j > ny) return;
                const int64_t d0 = pbase + noff[r];
                const bool ofixed = ((k == 0 ? (fixm >> 16) : fixm) >> r) & 1u;
                float sv[3] = {s.a.x, s.a.y, s.b};
                float xo[3] = {0.0f, 0.0f, 0.0f};
                if (ofixed || P.mode != EPI_RESID) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) xo[c] = __ldg(P.x + d0 + c);
                }
                if (ofixed) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) sv[c] = xo[c];
                }
                const int gs_c = P.mode - EPI_GS0 - 3 * node_colour(i, j, k);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float o;
                    if (P.mode == EPI_APPLY) {
                        o = sv[c];
                        if (want_dot) pdT += o * xo[c];
                    } else if (P.mode == EPI_RESID) {
                        o = __ldg(P.b + d0 + c) - sv[c];
                        if (want_dot) pdT += o * o;
                    } else if (P.mode == EPI_JACOBI) {
                        const float bb = __ldg(P.b + d0 + c);
                        o = xo[c] + omF * ((bb - sv[c]) * __ldg(P.idiag + d0 + c));
                        if (want_dot) pdT += o * bb;
                    } else if (P.mode == EPI_CHEB) {
                        const float bb = __ldg(P.b + d0 + c);
                        o = c0F * xo[c] + c2F * ((bb - sv[c]) * __ldg(P.idiag + d0 + c));
                        if (c1nz) o -= c1F * P.y[d0 + c];
                        if (want_dot) pdT += o * bb;
                    } else {
                        const float bb = __ldg(P.b + d0 + c);
                        o = gs_c == c ? xo[c] + (bb - sv[c]) * __ldg(P.idiag + d0 + c) : xo[c];
                        if (want_dot) pdT += o * bb;
                    }
                    P.y[d0 + c] = o;
                }
            };
            const V3 top = row_total(acc[NYB]);
            sy[k & 1][wid][lane] = make_float4(top.a.x, top.a.y, top.b, 0.0f);
#pragma unroll
            for (int r = 1; r < NYB; ++r) epilogue(r, row_total(acc[r]));
            V3 bot = row_total(acc[0]);
            __syncthreads();   // every warp's top row of plane k is in shared memory
            if (wid >= 1) {
                const float4 v = sy[k & 1][wid - 1][lane];
                bot = bot + V3{make_float2(v.x, v.y), v.z};
                epilogue(0, bot);
            }
        }
#pragma unroll
        for (int r = 0; r <= NYB; ++r) acc[r] = nxt[r];
    }

    // per-CTA partials; the last CTA finishes the dot and the alpha entry in a fixed order
    if (!want_dot && !P.with_alpha) return;
    const unsigned nblk = gridDim.x, blk = blockIdx.x;
    const int t = threadIdx.x;
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
    for (int q = t; q < int(nblk); q += NT) {
        td += ((volatile double*)P.partials)[q];
        ta += ((volatile double*)P.partials)[nblk + q];
    }
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
// plans: element rows per warp, warps per CTA, resident CTAs per SM asked of the register allocator
// ------------------------------------------------------------------------------------------------
#define PBM_STRIP_PLANS(X) \
    X(0, 4, 8, 1) X(1, 4, 4, 2) X(2, 3, 8, 1) X(3, 2, 8, 1) X(4, 2, 4, 2) X(5, 3, 4, 2)
#define PBM_STRIP_ROW(id, nyb, nw, minb) {nyb, nw, minb},
static const int kStripPlans[][3] = {PBM_STRIP_PLANS(PBM_STRIP_ROW)};
#undef PBM_STRIP_ROW
constexpr int kStripNumPlans = int(sizeof(kStripPlans) / sizeof(kStripPlans[0]));

int strip_num_plans() { return kStripNumPlans; }

int strip_threads(int cand) { return 32 * kStripPlans[cand][1]; }

FusedPlan strip_plan(const Geom& G, int cand) {
    FusedPlan p{};
    const int nyb = kStripPlans[cand][0], nw = kStripPlans[cand][1], per_sm = kStripPlans[cand][2];
    p.TX = kStripOwnedX;
    p.TY = nyb * nw - 1;
    p.gx = (G.nx + 1 + p.TX - 1) / p.TX;
    p.gy = (G.ny + 1 + p.TY - 1) / p.TY;
    const int planes = G.nz + 1;
    const int tiles = p.gx * p.gy;
    const int sms = num_sms();
    // a launch takes about waves x (DZ + 1) plane steps with per_sm resident CTAs per SM: the shortest, then the
    // fewest CTAs
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

template <int MODE>
static void strip_launch(int cand, int blocks, const StripArgs& P, cudaStream_t st) {
    switch (cand) {
#define PBM_STRIP_CASE(id, nyb, nw, minb) \
    case id: launch_pdl(k_strip_f32<MODE, nyb, nw, minb>, dim3(blocks), dim3(32 * nw), 0, st, P); break;
        PBM_STRIP_PLANS(PBM_STRIP_CASE)
#undef PBM_STRIP_CASE
        default: fail(PBM_EINVAL, "strip operator: unknown plan");
    }
}

void strip_fine_f32(int cand, const FusedPlan& p, const RedSet& r, const Geom& G, const KeHat& kh, const float* w,
                    const float* d, const float* u, const ApplyArgs& a, cudaStream_t st) {
    const bool s = d != nullptr;
    const int blocks = p.gx * p.gy * p.gz;
    if (2 * int64_t(blocks) > r.len) fail(PBM_EINVAL, "grid too large for the partials buffer");
    StripArgs P{};
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.support = G.support;
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
    if (s) strip_launch<2>(cand, blocks, P, st);
    else strip_launch<0>(cand, blocks, P, st);
    PBM_LAUNCH("strip FP32 fine operator");
}

}  // namespace pbm
