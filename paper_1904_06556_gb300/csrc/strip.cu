// Single-pass FP32 fine-level operator in lane strips: K(w) x and the S operator of eq. (S) with the fused
// apply / residual / damped-Jacobi / Chebyshev / Gauss-Seidel epilogues (Section 5.1) and the Krylov dot
// products, organised so that almost every value an element shares with its neighbours stays in registers and
// every floating-point instruction does the work of two elements.
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
// Two vertically adjacent elements of the strip are processed together: every per-element quantity is a float2
// (lower element, upper element), so the paired FP32 instructions (FADD2 / FMUL2 / FFMA2) do all arithmetic of
// the transform and of Khat for both at once. The output goes back the same way: each element's bottom face
// plus the top face of the element below it in the previous layer (carried in transformed form) is split into
// the x-pair form of its two node rows, and a node's value is its own column's part plus the part the lane on
// its left computed (one shuffle per value). The node row between two warps is completed through shared memory
// (one float4 per lane and plane), handed from the lower warp to the upper one with a pair of named barriers, so
// that every warp waits only for its neighbours. Nothing but the
// inputs and the output goes through global memory, and no element value is recomputed except on the CTA's
// one-column and one-row halo and on the layer below each plane chunk.
//
// The alpha row of S counts every element once (in the CTA and chunk that own its upper corner node). Per-CTA
// partial sums of the dot product and of the alpha row are finished by the last CTA in a fixed order, so the
// results are bit-reproducible for a given plan.
#include <algorithm>
#include <atomic>

#include "fp32_elem.h"
#include "pbm_internal.h"

namespace pbm {

namespace {

constexpr int kStripOwnedX = 30;   // owned node columns per warp (lanes 1 .. 30)

// Khat of pbm_internal.h with every coefficient repeated in both halves of a float2 (the two elements of a pair)
struct KeHatP {
    float2 dg[3][8];
    float2 lam4[2];
    float2 mu4[2];
};

// Y = Khat X for two elements at once (X, Y: [component][pattern], patterns 1 .. 7; Y[.][0] is zero)
__device__ __forceinline__ void khat_pair(const KeHatP& K, const float2 (&X)[3][8], float2 (&Y)[3][8]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Y[c][0] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            float2 acc = mul2(K.dg[c][q], X[c][q]);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d == c) continue;
                const int r = 3 - c - d;
                const int br = (q >> r) & 1;
                const int qc = (q >> c) & 1, qd = (q >> d) & 1;
                if (qc == 1 && qd == 0) acc = fma2(K.lam4[br], X[d][(q & ~(1 << c)) | (1 << d)], acc);
                if (qd == 1 && qc == 0) acc = fma2(K.mu4[br], X[d][(q & ~(1 << d)) | (1 << c)], acc);
            }
            Y[c][q] = acc;
        }
    }
}

// face quads of the two elements of a pair on one plane, per pattern q and component c, as (lower element, upper
// element): fused.cu's convention, q = 0 sum, 1 x-difference, 2 y-difference, 3 both
struct FQ {
    float2 q[4][3];
};

// the 24 transformed coefficients of the two elements from the face quads of their bottom and top planes
__device__ __forceinline__ void pair_coeffs(const FQ& b, const FQ& t, float2 (&X)[3][8]) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            X[c][q] = add2(b.q[q][c], t.q[q][c]);
            X[c][q + 4] = sub2(t.q[q][c], b.q[q][c]);
        }
}

// 4-byte asynchronous global -> shared copy, the bytes beyond src_bytes (0 or 4) zero-filled
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// named barriers between two adjacent warps (64 threads): one warp waits, the other arrives
__device__ __forceinline__ void bar_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id) { asm volatile("bar.arrive %0, 64;" ::"r"(id) : "memory"); }

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Layout of a lane's staging ring (floats per stage, in units of the CTA's thread count): x of node rows 0 .. NYB
// (and u for S), the element weights of NYB rows (and the Schur weights for S), then NE epilogue operands of the
// owned node rows 0 .. NYB - 1 (b; the inverse diagonal; the previous Chebyshev iterate). D stages: as many as
// fit MINB CTAs per SM (5 or 4 for plain applies, at least 3).
struct StripRing {
    int D, NV, WOFF, EOFF, NE, PER;
};
__host__ __device__ constexpr int strip_epi_operands(int epi) {
    return epi == EPI_APPLY ? 0 : (epi == EPI_RESID ? 1 : (epi == EPI_CHEB ? 3 : 2));
}
__host__ __device__ constexpr StripRing strip_ring(int mode, int epi, int nyb, int nw, int minb) {
    const bool s = mode == 2;
    const int nv = 3 * (nyb + 1);
    const int woff = s ? 2 * nv : nv;
    const int eoff = woff + (s ? 2 * nyb : nyb);
    const int ne = strip_epi_operands(epi);
    const int per = eoff + 3 * nyb * ne;
    int d = s ? 4 : 5;
    // shared memory per SM: 228 KB, less about 3 KB per CTA for the static arrays and the reserved block
    while (d > 3 && minb * (d * per * 32 * nw * 4 + 3 * 1024) > 228 * 1024) --d;
    return StripRing{d, nv, woff, eoff, ne, per};
}

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
    KeHatP K;
    double* partials;     // 2 * gridDim.x
    DevScalars* sc;
    unsigned int* counter;
};

}  // namespace

// MODE 0: K(w) x. MODE 2: S x with W_e = Khat H u_e recomputed from u. EPI: the epilogue (EPI_APPLY, EPI_RESID,
// EPI_JACOBI, EPI_CHEB, or EPI_GS0 for every Gauss-Seidel colour, the colour read from P.mode). NW warps per CTA,
// NYB (even) element rows per warp, MINB resident CTAs per SM asked of the register allocator.
template <int MODE, int EPI, int NYB, int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) k_strip_f32(StripArgs P) {
    pdl_wait();
    constexpr bool S = MODE == 2;
    constexpr int NT = 32 * NW;
    constexpr int R = NW * NYB;            // element rows of the CTA
    constexpr int NP = NYB / 2;            // element pairs per lane
    static_assert(NYB % 2 == 0, "element rows come in pairs");
    // the face quads of a layer's upper plane are kept for the next layer where the registers allow it (one pair
    // per lane, and for S only with the two 4-warp CTAs per SM); otherwise every layer transforms both planes
    constexpr bool CARRY = NP == 1 && (!S || (NW == 4 && MINB == 2));
    __shared__ float4 sy[NW][32];          // node totals of each warp's top row for the warp above
    static_assert(2 * NW - 2 <= 15, "named barriers: 1 .. NW - 1 (row written), NW .. 2 NW - 2 (row read)");
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

    // node rows r = 0 .. NYB: in range and not supported (bit r for planes k >= 1, bit 16 + r for plane 0),
    // supported (same layout), owned by this lane (bit r)
    unsigned okm = 0, fixm = 0, ownm = 0, inm = 0;
    int noff[NYB + 1];                     // node offsets (floats) within a plane
    const int ic = min(max(i, 0), nx);     // clamped coordinates: every address formed stays inside the arrays
#pragma unroll
    for (int r = 0; r <= NYB; ++r) {
        const int j = jb + r;
        const bool in = i >= 0 && i <= nx && j >= 0 && j <= ny;
        noff[r] = 3 * (ic + (nx + 1) * min(max(j, 0), ny));
        if (in) {
            inm |= 1u << r;
            const int fb = fixed_bits(support, nx, ny, nz, i, j);
            if (!(fb & 1)) okm |= 1u << r;
            if (!(fb & 2)) okm |= 1u << (16 + r);
            fixm |= unsigned(fb & 1) << r;
            fixm |= unsigned((fb >> 1) & 1) << (16 + r);
            if (lane >= 1 && lane <= 30 && r < NYB && (r >= 1 || wid >= 1)) ownm |= 1u << r;
        }
    }
    // element rows r = 0 .. NYB - 1 that exist (lanes 0 .. 30), and those whose alpha term this CTA counts
    unsigned em = 0, am = 0;
    int eoff[NYB];
#pragma unroll
    for (int r = 0; r < NYB; ++r) {
        const int j = jb + r;
        const bool e = lane <= 30 && i >= 0 && i < nx && j >= 0 && j < ny;
        eoff[r] = min(max(i, 0), nx - 1) + nx * min(max(j, 0), ny - 1);
        if (e) em |= 1u << r;
        if (e && lane >= 1 && j >= Y0) am |= 1u << r;
    }

    const float xa = S ? P.x[P.n] : 0.0f;
    float omF = 0.0f, c0F = 0.0f, c1F = 0.0f, c2F = 0.0f;
    bool c1nz = false;
    if (EPI == EPI_JACOBI) omF = float(*P.omega);
    if (EPI == EPI_CHEB) {
        c0F = float(P.omega[0]);
        c1F = float(P.omega[1]);
        c2F = float(P.omega[2]);
        c1nz = c1F != 0.0f;
    }
    const bool want_dot = P.dot_slot >= 0;
    float pdT = 0.0f, paT = 0.0f;

    // Asynchronous staging (cp.async): every lane copies its own column's values into a private ring of D stages
    // in shared memory. Stage p holds x (and u) of plane p, rows 0 .. NYB (zero where not in range or supported,
    // by the copies' zero fill), and the weights of layer p - 1. Layer k reads planes k and k + 1 from the ring
    // (both stay resident while it runs, so no plane's transform is kept in registers across layers) and then
    // issues plane k + D - 1 into the slot of plane k - 1. A lane only reads what it copied itself, so waiting for
    // its own copies suffices (no barrier).
    constexpr StripRing RG = strip_ring(MODE, EPI, NYB, NW, MINB);
    constexpr int D = RG.D, NV = RG.NV, WOFF = RG.WOFF, EOFF = RG.EOFF, PER = RG.PER;
    extern __shared__ float ring[];   // D * PER * NT floats (dynamic: strip_ring_bytes)
    const int tid = threadIdx.x;
    const int pmax = min(kz1, nz);   // last plane a layer of this chunk reads
    const uint32_t ring0 = uint32_t(__cvta_generic_to_shared(ring + tid));
    int islot = 0;   // ring slot of the next stage issued
    auto issue = [&](int p) {
        if (p <= pmax) {
            const uint32_t st = ring0 + uint32_t(islot * PER * NT * 4);
            const unsigned ok = p == 0 ? (okm >> 16) : okm;
            const float* xs = P.x + int64_t(p) * plane;
            const float* us = S ? P.u + int64_t(p) * plane : nullptr;
#pragma unroll
            for (int r = 0; r <= NYB; ++r) {
                const uint32_t nb = ((ok >> r) & 1u) ? 4u : 0u;   // zero fill where not in range or supported
                const float* xr = xs + noff[r];
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_async4(st + 4u * uint32_t((3 * r + c) * NT), xr + c, nb);
                if (S) {
                    const float* ur = us + noff[r];
#pragma unroll
                    for (int c = 0; c < 3; ++c) cp_async4(st + 4u * uint32_t((NV + 3 * r + c) * NT), ur + c, nb);
                }
            }
            if (RG.NE > 0) {
                // the epilogue's operands of the owned node rows 0 .. NYB - 1 of plane p (zero outside the grid; the
                // previous Chebyshev iterate only when its coefficient is not zero)
                const float* bs = P.b + int64_t(p) * plane;
                const float* ds = RG.NE >= 2 ? P.idiag + int64_t(p) * plane : nullptr;   // only where staged
                const float* ys = RG.NE >= 3 ? P.y + int64_t(p) * plane : nullptr;
#pragma unroll
                for (int r = 0; r < NYB; ++r) {
                    const uint32_t nb = ((inm >> r) & 1u) ? 4u : 0u;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        cp_async4(st + 4u * uint32_t((EOFF + 3 * r + c) * NT), bs + noff[r] + c, nb);
                        if (RG.NE >= 2)
                            cp_async4(st + 4u * uint32_t((EOFF + 3 * (NYB + r) + c) * NT), ds + noff[r] + c, nb);
                        if (RG.NE >= 3)
                            cp_async4(st + 4u * uint32_t((EOFF + 3 * (2 * NYB + r) + c) * NT), ys + noff[r] + c,
                                      c1nz ? nb : 0u);
                    }
                }
            }
            if (p >= 1) {
                const float* wl = P.w + int64_t(p - 1) * elayer;
                const float* dl = S ? P.d + int64_t(p - 1) * elayer : nullptr;
#pragma unroll
                for (int r = 0; r < NYB; ++r) {
                    const uint32_t nb = ((em >> r) & 1u) ? 4u : 0u;
                    cp_async4(st + 4u * uint32_t((WOFF + r) * NT), wl + eoff[r], nb);
                    if (S) cp_async4(st + 4u * uint32_t((WOFF + NYB + r) * NT), dl + eoff[r], nb);
                }
            }
        }
        cp_async_commit();
        islot = islot == D - 1 ? 0 : islot + 1;
    };
    // raw values of plane p and the weights of layer p - 1, from the lane's ring
    float rx[NYB + 1][3], ru[NYB + 1][3];   // ru: S only (dead code for K)
    float2 wn[NP], dn[NP];
    auto read_plane = [&](int slot) {
        const float* st = ring + slot * PER * NT + tid;
#pragma unroll
        for (int r = 0; r <= NYB; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rx[r][c] = st[(3 * r + c) * NT];
                if (S) ru[r][c] = st[(NV + 3 * r + c) * NT];
            }
    };
    auto read_w = [&](int slot) {
        const float* st = ring + slot * PER * NT + tid;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            wn[q] = make_float2(st[(WOFF + 2 * q) * NT], st[(WOFF + 2 * q + 1) * NT]);
            if (S) dn[q] = make_float2(st[(WOFF + NYB + 2 * q) * NT], st[(WOFF + NYB + 2 * q + 1) * NT]);
        }
    };
    int cslot = 0;   // ring slot of plane k of the current layer

    // face quads of a plane from the lane's raw column values and the right neighbour's: the x-pairs (sum and
    // difference of the two node columns) of the element pair's low rows (2p, 2p + 1) and high rows (2p + 1, 2p + 2),
    // then their sum and difference along y
    auto plane_quads = [&](const float (&v)[NYB + 1][3], FQ (&o)[NP]) {
        float rt[NYB + 1][3];
#pragma unroll
        for (int r = 0; r <= NYB; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) rt[r][c] = shfl_dn1(v[r][c]);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 ownL = make_float2(v[2 * p][c], v[2 * p + 1][c]);
                const float2 ownH = make_float2(v[2 * p + 1][c], v[2 * p + 2][c]);
                const float2 rgtL = make_float2(rt[2 * p][c], rt[2 * p + 1][c]);
                const float2 rgtH = make_float2(rt[2 * p + 1][c], rt[2 * p + 2][c]);
                const float2 ls = add2(rgtL, ownL), ld = sub2(rgtL, ownL);
                const float2 hs = add2(rgtH, ownH), hd = sub2(rgtH, ownH);
                o[p].q[0][c] = add2(ls, hs);
                o[p].q[1][c] = add2(ld, hd);
                o[p].q[2][c] = sub2(hs, ls);
                o[p].q[3][c] = sub2(hd, ld);
            }
    };

    // epilogue of the node of row r of plane k with the operator value s: stored (and counted in the dot) where
    // the lane owns it; the loads use the clamped, always valid addresses, so no lane branches
    // epilogue of the node of row r of plane k with the operator value s: stored (and counted in the dot) where
    // the lane owns it. x and the epilogue's operands come from the lane's ring stage of plane k (slot es); x is
    // zero there at supported nodes, whose output is x itself, read from global memory (predicated: only lanes of
    // supported nodes load). The store uses the clamped, always valid address, so no lane branches.
    auto epilogue = [&](int es, int k, int r, float s0, float s1, float s2) {
        const bool own = (ownm >> r) & 1u;
        const int j = jb + r;
        const int64_t d0 = int64_t(k) * plane + noff[r];
        const bool ofixed = ((k == 0 ? (fixm >> 16) : fixm) >> r) & 1u;
        const float* st = ring + es * PER * NT + tid;
        float sv[3] = {s0, s1, s2};
        float xo[3] = {0.0f, 0.0f, 0.0f};
        constexpr bool always_x = EPI == EPI_JACOBI || EPI == EPI_CHEB || EPI == EPI_GS0;
        if (always_x || (EPI == EPI_APPLY && want_dot)) {
#pragma unroll
            for (int c = 0; c < 3; ++c) xo[c] = st[(3 * r + c) * NT];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (ofixed) xo[c] = __ldg(P.x + d0 + c);   // supported nodes only
            sv[c] = ofixed ? xo[c] : sv[c];
        }
        const int gs_c = EPI == EPI_GS0 ? P.mode - EPI_GS0 - 3 * node_colour(i, j, k) : 0;
        float dsum = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float o;
            if (EPI == EPI_APPLY) {
                o = sv[c];
                dsum += o * xo[c];
            } else if (EPI == EPI_RESID) {
                o = st[(EOFF + 3 * r + c) * NT] - sv[c];
                dsum += o * o;
            } else if (EPI == EPI_JACOBI) {
                const float bb = st[(EOFF + 3 * r + c) * NT];
                o = xo[c] + omF * ((bb - sv[c]) * st[(EOFF + 3 * (NYB + r) + c) * NT]);
                dsum += o * bb;
            } else if (EPI == EPI_CHEB) {
                const float bb = st[(EOFF + 3 * r + c) * NT];
                o = c0F * xo[c] + c2F * ((bb - sv[c]) * st[(EOFF + 3 * (NYB + r) + c) * NT]);
                o -= c1F * st[(EOFF + 3 * (2 * NYB + r) + c) * NT];   // staged as zero when c1 is zero
                dsum += o * bb;
            } else {
                const float bb = st[(EOFF + 3 * r + c) * NT];
                o = gs_c == c ? xo[c] + (bb - sv[c]) * st[(EOFF + 3 * (NYB + r) + c) * NT] : xo[c];
                dsum += o * bb;
            }
            if (own) P.y[d0 + c] = o;
        }
        if (want_dot && own) pdT += dsum;
    };

    // One layer k (planes k and k + 1): xlo / ulo hold the face quads of plane k (x and u), carry the
    // transformed top faces of layer k - 1 (zero below the first layer); xhi / uhi receive those of plane k + 1,
    // which the next layer takes as its lo, and carry the top faces of layer k. Then the node values of plane k
    // are finished (k >= kz0). Called with the lo / hi roles swapped on alternate layers, so every plane is read
    // from the ring and transformed once and nothing is copied between layers.
    auto layer_step = [&](int k, float2 (&carry)[NP][4][3], FQ (&xlo)[NP], FQ (&ulo)[NP], FQ (&xhi)[NP],
                          FQ (&uhi)[NP]) {
        const bool layer = k < nz;
        // node-row accumulators of plane k: the left (own column) and right (next column) parts per component,
        // rows 0 .. NYB
        float aL[NYB + 1][3], aR[NYB + 1][3];
#pragma unroll
        for (int r = 0; r <= NYB; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) aL[r][c] = aR[r][c] = 0.0f;
        // a face of element pair p (transformed, 4 q-values per element) split into its low and high node rows and
        // into the left and right columns: low row (F0 - F2) -/+ (F1 - F3), high row (F0 + F2) -/+ (F1 + F3)
        auto face_rows = [&](float2 F0, float2 F1, float2 F2, float2 F3, int p, int c) {
            const float2 ls = sub2(F0, F2), ld = sub2(F1, F3);
            const float2 hs = add2(F0, F2), hd = add2(F1, F3);
            const float2 lL = sub2(ls, ld), lR = add2(ls, ld), hL = sub2(hs, hd), hR = add2(hs, hd);
            aL[2 * p][c] += lL.x;
            aR[2 * p][c] += lR.x;
            aL[2 * p + 1][c] += hL.x + lL.y;
            aR[2 * p + 1][c] += hR.x + lR.y;
            aL[2 * p + 2][c] += hL.y;
            aR[2 * p + 2][c] += hR.y;
        };
        const int es = cslot;   // ring slot of plane k: its epilogue operands
        const int hslot = cslot == D - 1 ? 0 : cslot + 1;
        if (layer) {
            cp_async_wait<D - 3>();  // plane k + 1 and the weights of layer k have landed
            if (!CARRY) {
                read_plane(cslot);
                plane_quads(rx, xlo);
                if (S) plane_quads(ru, ulo);
            }
            read_plane(hslot);
            read_w(hslot);
            plane_quads(rx, xhi);
            if (S) plane_quads(ru, uhi);
            const float2 (&we)[NP] = wn;
            const float2 (&de)[NP] = dn;
            const bool count_alpha = k + 1 >= kz0 && k + 1 < kz1;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 X[3][8], Y[3][8];
                pair_coeffs(xlo[p], xhi[p], X);
                if (S) {
                    // t_e = d_e (u_e^T K_e x_e - x_alpha) with u_e^T K_e x_e = (H u_e) . Khat (H x_e); then
                    // Y = Khat (w_e X + t_e H u_e) (linearity: the two products of eq. (S) share one Khat)
                    float2 U[3][8];
                    pair_coeffs(ulo[p], uhi[p], U);
                    khat_pair(P.K, X, Y);
                    float2 dc[3];   // one partial sum per component: short dependency chains
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        dc[c] = mul2(U[c][1], Y[c][1]);
#pragma unroll
                        for (int q = 2; q < 8; ++q) dc[c] = fma2(U[c][q], Y[c][q], dc[c]);
                    }
                    const float2 dot = add2(add2(dc[0], dc[1]), dc[2]);
                    const float2 te = mul2(de[p], make_float2(dot.x - xa, dot.y - xa));
                    if (count_alpha) {
                        if ((am >> (2 * p)) & 1u) paT -= te.x;
                        if ((am >> (2 * p + 1)) & 1u) paT -= te.y;
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int q = 1; q < 8; ++q) X[c][q] = fma2(te, U[c][q], mul2(we[p], X[c][q]));
                    khat_pair(P.K, X, Y);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        // bottom face plus the carried top face of the layer below; the new top face is carried
                        float2 F[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            F[q] = add2(carry[p][q][c], sub2(Y[c][q], Y[c][q + 4]));
                            carry[p][q][c] = add2(Y[c][q], Y[c][q + 4]);
                        }
                        face_rows(F[0], F[1], F[2], F[3], p, c);
                    }
                } else {
                    khat_pair(P.K, X, Y);
                    // the element weight enters with the faces: top w (Y_q + Y_q+4), bottom plus carry
                    // carry + w (Y_q - Y_q+4); Y_0 = 0
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float2 F[4];
                        const float2 wy4 = mul2(we[p], Y[c][4]);
                        F[0] = sub2(carry[p][0][c], wy4);
                        carry[p][0][c] = wy4;
#pragma unroll
                        for (int q = 1; q < 4; ++q) {
                            const float2 wyq4 = mul2(we[p], Y[c][q + 4]);
                            F[q] = sub2(fma2(we[p], Y[c][q], carry[p][q][c]), wyq4);
                            carry[p][q][c] = fma2(we[p], Y[c][q], wyq4);
                        }
                        face_rows(F[0], F[1], F[2], F[3], p, c);
                    }
                }
            }
            issue(k + D - 1);        // into the slot of plane k - 1
        } else {
            // above the last layer: plane k = nz holds only the top faces of layer nz - 1
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int c = 0; c < 3; ++c) face_rows(carry[p][0][c], carry[p][1][c], carry[p][2][c], carry[p][3][c], p, c);
        }
        cslot = hslot;
        if (k < kz0) return;   // the layer below the chunk: only its top faces are kept
        // node totals: the own column's left part plus the left lane's right part
        float tot[NYB + 1][3];
#pragma unroll
        for (int r = 0; r <= NYB; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) tot[r][c] = aL[r][c] + shfl_up1(aR[r][c]);
        // the top row goes to the warp above through its slot: wait until that warp has read the previous plane's
        // value, write, signal; rows 1 .. NYB - 1 meanwhile; then the bottom row from the warp below
        if (wid + 1 < NW) {
            bar_sync(NW + wid);
            sy[wid][lane] = make_float4(tot[NYB][0], tot[NYB][1], tot[NYB][2], 0.0f);
            bar_arrive(1 + wid);
        }
#pragma unroll
        for (int r = 1; r < NYB; ++r) epilogue(es, k, r, tot[r][0], tot[r][1], tot[r][2]);
        if (wid >= 1) {
            bar_sync(1 + wid - 1);
            const float4 v = sy[wid - 1][lane];
            bar_arrive(NW + wid - 1);
            epilogue(es, k, 0, tot[0][0] + v.x, tot[0][1] + v.y, tot[0][2] + v.z);
        }
    };

    const int kstart = max(kz0 - 1, 0);
    float2 carry[NP][4][3];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) carry[p][q][c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < D - 1; ++q) issue(kstart + q);
    // the slot between warps w and w + 1 starts free: the reader's first "read done" is signalled up front, and
    // the writer's last wait matches the reader's last signal, so every barrier phase completes
    if (wid >= 1) bar_arrive(NW + wid - 1);
    // face quads of the first plane; from then on every layer transforms only its upper plane
    FQ xa_[NP], ua_[NP], xb_[NP], ub_[NP];   // ua_, ub_: S only
    cp_async_wait<D - 2>();
    read_plane(0);
    plane_quads(rx, xa_);
    if (S) plane_quads(ru, ua_);
    for (int k = kstart; k < kz1; k += 2) {
        layer_step(k, carry, xa_, ua_, xb_, ub_);
        if (k + 1 < kz1) layer_step(k + 1, carry, xb_, ub_, xa_, ua_);
    }
    if (wid + 1 < NW) bar_sync(NW + wid);
    cp_async_wait<0>();

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
    td = l2_strided_sum(P.partials, int(nblk), t, NT);
    ta = l2_strided_sum(P.partials + nblk, int(nblk), t, NT);
    double sd = fused_cta_sum<NT>(td, sred);
    const double sa = fused_cta_sum<NT>(ta, sred);
    if (t != 0) return;
    *P.counter = 0u;
    if (P.with_alpha) {
        const int64_t n = P.n;
        double o;
        if (EPI == EPI_APPLY) {
            o = sa;
            sd += o * double(xa);
        } else if (EPI == EPI_RESID) {
            o = double(P.b[n]) - sa;
            sd += o * o;
        } else if (EPI == EPI_JACOBI) {
            const double bb = double(P.b[n]);
            o = double(xa) + *P.omega * ((bb - sa) * double(P.idiag[n]));
            sd += o * bb;
        } else if (EPI == EPI_CHEB) {
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
#define PBM_STRIP_PLANS(X) X(0, 2, 4, 2) X(1, 2, 8, 2) X(2, 2, 4, 3) X(3, 2, 6, 2)
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
    // a launch takes about waves x (DZ + 1) plane steps with per_sm resident CTAs per SM: the shortest, and of
    // equally short ones the one with the fewest CTAs (the least halo work)
    double best = 1e300;
    p.DZ = planes;
    for (int dz = std::max(1, std::min(planes, 2)); dz <= planes; ++dz) {
        const int gz = (planes + dz - 1) / dz;
        if (dz > 1 && (planes + dz - 2) / (dz - 1) == gz && dz != planes) continue;
        const double waves = double((int64_t(tiles) * gz + sms * per_sm - 1) / (sms * per_sm));
        const double cost = waves * (dz + 1);
        if (cost <= best + 1e-9) {
            best = cost;
            p.DZ = dz;
        }
    }
    p.gz = (planes + p.DZ - 1) / p.DZ;
    return p;
}

// bytes of the staging ring of the kernel: D stages of x (and u) of NYB + 1 node rows, the weights of NYB element
// rows and the epilogue's operands, per thread
static size_t strip_ring_bytes(int mode, int epi, int nyb, int nw, int minb) {
    const StripRing rg = strip_ring(mode, epi, nyb, nw, minb);
    return sizeof(float) * size_t(rg.D) * size_t(rg.PER) * size_t(32 * nw);
}

// launch with the ring in dynamic shared memory (the opt-in above 48 KB set once per kernel and device)
template <int MODE, int EPI, int NYB, int NW, int MINB>
static void strip_launch_one(int blocks, const StripArgs& P, cudaStream_t st) {
    auto kern = k_strip_f32<MODE, EPI, NYB, NW, MINB>;
    const size_t smem = strip_ring_bytes(MODE, EPI, NYB, NW, MINB);
    static std::atomic<uint64_t> set_on{0};   // bit per device ordinal < 64
    int dev = 0;
    PBM_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (!bit || !(set_on.load() & bit)) {
        PBM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        if (bit) set_on.fetch_or(bit);
    }
    launch_pdl(kern, dim3(blocks), dim3(32 * NW), smem, st, P);
}

template <int MODE, int EPI>
static void strip_launch_epi(int cand, int blocks, const StripArgs& P, cudaStream_t st) {
    switch (cand) {
#define PBM_STRIP_CASE(id, nyb, nw, minb) \
    case id: strip_launch_one<MODE, EPI, nyb, nw, minb>(blocks, P, st); break;
        PBM_STRIP_PLANS(PBM_STRIP_CASE)
#undef PBM_STRIP_CASE
        default: fail(PBM_EINVAL, "strip operator: unknown plan");
    }
}

template <int MODE>
static void strip_launch(int cand, int blocks, const StripArgs& P, cudaStream_t st) {
    switch (P.mode) {
        case EPI_APPLY: strip_launch_epi<MODE, EPI_APPLY>(cand, blocks, P, st); break;
        case EPI_RESID: strip_launch_epi<MODE, EPI_RESID>(cand, blocks, P, st); break;
        case EPI_JACOBI: strip_launch_epi<MODE, EPI_JACOBI>(cand, blocks, P, st); break;
        case EPI_CHEB: strip_launch_epi<MODE, EPI_CHEB>(cand, blocks, P, st); break;
        default:
            if (P.mode < EPI_GS0 || P.mode > EPI_GS0 + kGsColours) fail(PBM_EINVAL, "strip operator: unknown epilogue");
            strip_launch_epi<MODE, EPI_GS0>(cand, blocks, P, st);
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
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 8; ++q) P.K.dg[c][q] = make_float2(float(kh.dg[c][q]), float(kh.dg[c][q]));
    for (int b = 0; b < 2; ++b) {
        P.K.lam4[b] = make_float2(float(kh.lam4[b]), float(kh.lam4[b]));
        P.K.mu4[b] = make_float2(float(kh.mu4[b]), float(kh.mu4[b]));
    }
    P.partials = r.partials;
    P.sc = r.sc;
    P.counter = r.counter;
    if (s) strip_launch<2>(cand, blocks, P, st);
    else strip_launch<0>(cand, blocks, P, st);
    PBM_LAUNCH("strip FP32 fine operator");
}

}  // namespace pbm
