// Tensor-core variant of the single-pass FP32 fine-level operator: K(w) x and the S operator of
// eq. (S) (Section 5.1) with the element contraction y_e = K_e x_e on the tcgen05 tensor cores.
//
// The march is that of the CUDA-core kernel (fused.cu): a CTA owns 31 x 7 node columns, computes the
// 32 x 8 element columns around them and marches up a chunk of node planes; the four element columns
// around a node are summed in a fixed order by the thread that owns it, which applies the epilogue.
// What changes is the element arithmetic. One element layer of the tile is the product
//     D = X K^T,   X: 256 elements x 32,   K: the 24 x 24 element matrix padded to 32 x 32,
// issued as two M = 128, N = 32 MMAs (accumulator in tensor memory), where row e of X holds the
// element's 8 corner nodes as (x, y, z, 0) and the padding of K is a zero row and column after every
// third entry. X is never copied per element: the staged node plane keeps, for every element row
// and every run of 8 elements along x, the 9 nodes of that run as float4 (a node shared by two runs
// is stored twice). The 8 rows of one core matrix of the operand (8 consecutive elements, 16 bytes
// each) are then 8 consecutive node slots, the next 8 rows start 9 slots later (SBO = 144 bytes), and
// the corner one node further along x is the next slot (LBO = 16 bytes), so the MMA reads the
// corners of the 128 elements of one operand straight from the staged plane. The four (y, z) corner
// pairs are the four K steps of 8.
//
// Precision: TF32 keeps 11 significant bits. Every staged value is stored as hi = x rounded to TF32
// and lo = x - hi, and D = hi K + lo K (+ hi K_lo when K itself is not exact in TF32), which bounds
// the product error by about 2^-23 |x| |K|, the rounding of FP32 arithmetic. For the isotropic cube
// K_e is a multiple of a matrix of small integers whenever nu is a simple fraction (for nu = 0.3,
// 88 K_e / K_e[0][0] is an integer matrix), and then only x is split: two terms, not three.
//
// Pipeline (one __syncthreads per layer): while the CUDA cores of the CTA turn layer k's
// accumulator into node sums, the tensor core already runs layer k + 1 into the other accumulator
// buffer; planes are staged three ahead into a ring of four and the plane after that is prefetched
// into registers. Every wait on the tensor core is bounded: a wait that gives up sets flags[4] of the
// device scalars, poisons the output with a NaN, and the CTA frees its tensor memory and returns.
#include <cmath>
#include <cstring>

#include "pbm_internal.h"

namespace pbm {

namespace tc {
constexpr int NT = 256;             // 8 warps: warp w computes element row w of the tile
constexpr int EXT = 32, EYT = 8;    // element columns of a tile
constexpr int TX = EXT - 1, TY = EYT - 1;   // owned node columns
constexpr int SEG = EXT / 8;        // runs of 8 elements per element row
constexpr int NROW = EYT + 1;       // staged node rows
constexpr int SLOTS = NROW * SEG * 9;   // float4 node slots of one staged plane
constexpr int RING = 4;             // staged planes
constexpr int PSLOT = 2;            // staging slots per thread
constexpr int BFLOATS = 1024;       // one 32 x 32 operand matrix
static_assert(SLOTS <= PSLOT * NT, "staging slots");
}  // namespace tc

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major,
// N / 8 in bits 17-22, M / 16 in bits 24-28; M = 128, N = 32
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t pack_desc(uint32_t lo, uint32_t hi) { return (uint64_t(hi) << 32) | lo; }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes of shared memory made visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    // suspend-time hint 1 ms: the thread sleeps until the phase completes or the hint runs out
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}

// waits for the completion of phase `parity` of the mbarrier at shared address a, for one second at
// most (then false)
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = gtimer();
    while (gtimer() - t0 < 1000000000ull)
        if (mbar_try(a, parity)) return true;
    return false;
}

// 32 consecutive accumulator columns of this thread's lane (the wait is part of the same asm, so no
// use of the registers can be scheduled before the data has arrived)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x rounded to the nearest TF32 value (ties away from zero): half a unit of the 11th significant bit
// added to the magnitude, the 13 bits below it cleared (finite x far below the FP32 maximum)
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void split_store(float4* hi, float4* lo, const float (&v)[3], bool zero) {
    const float a = zero ? 0.0f : v[0], b = zero ? 0.0f : v[1], c = zero ? 0.0f : v[2];
    const float ha = tf32_hi(a), hb = tf32_hi(b), hc = tf32_hi(c);
    *hi = make_float4(ha, hb, hc, 0.0f);
    *lo = make_float4(a - ha, b - hb, c - hc, 0.0f);
}

template <int NT>
__device__ __forceinline__ double tc_cta_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

}  // namespace

struct TcArgs {
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
    int terms;            // MMA terms per K step: 2 (element matrix exact in TF32) or 3
    float kscale;         // K_e = kscale x (the matrix of B)
    const float* B;       // [2][1024]: hi and lo parts of the scaled element matrix in the operand layout
    double* partials;     // 2 * gridDim.x
    DevScalars* sc;
    unsigned int* counter;
};

// MODE 0: K(w) x. MODE 2: S x, with W_e = K_e u_e from a second product on the staged u.
template <int MODE, int MINB>
__global__ void __launch_bounds__(tc::NT, MINB) k_tc_f32(TcArgs P) {
    using namespace tc;
    pdl_wait();
    constexpr bool S = MODE == 2;
    constexpr int NV = S ? 2 : 1;                  // staged vectors: x (and u)
    constexpr uint32_t NCOL = S ? 256 : 128;       // 2 buffers x 2 MMA halves x NV x 32 columns
    constexpr int PL = 2 * SLOTS;                  // float4 per staged plane (hi, lo)
    extern __shared__ float4 tc_sm[];
    float4* stg = tc_sm;                           // [NV][RING][hi, lo][SLOTS]
    float4* sB = stg + NV * RING * PL;             // [hi, lo][256]
    float4* sq = sB + 2 * (BFLOATS / 4);           // [2][EYT][EXT] row sums of the node exchange
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ double sred[NT / 32];
    __shared__ int s_abort;
    __shared__ bool s_last;

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int nx = P.nx, ny = P.ny, nz = P.nz, support = P.support;
    const int bx = int(blockIdx.x % unsigned(P.gx));
    const int rest = int(blockIdx.x / unsigned(P.gx));
    const int by = rest % P.gy, bz = rest / P.gy;
    const int X0 = bx * TX, Y0 = by * TY;
    const int kz0 = bz * P.DZ, kz1 = min(kz0 + P.DZ, nz + 1);
    const int64_t plane = 3 * int64_t(nx + 1) * (ny + 1);
    const int kstart = max(kz0 - 1, 0);
    const int pmax = min(kz1, nz);                 // last node plane the chunk reads

    // staging slots q = t + s NT (node row j, run r, node i of the run): a pointer to the node in the
    // next plane to fetch, and whether the node is in the grid / supported on plane 0 / on the others
    const float* gx[PSLOT];
    const float* gu[PSLOT];
    unsigned has = 0, in = 0, fix0 = 0, fix1 = 0;
#pragma unroll
    for (int s = 0; s < PSLOT; ++s) {
        const int q = t + s * NT;
        int64_t o = 0;
        if (q < SLOTS) {
            has |= 1u << s;
            const int j = q / (SEG * 9), rr = q - j * (SEG * 9);
            const int run = rr / 9, i = rr - run * 9;
            const int gxn = X0 - 1 + 8 * run + i, gyn = Y0 - 1 + j;
            if (gxn >= 0 && gxn <= nx && gyn >= 0 && gyn <= ny) {
                in |= 1u << s;
                o = 3 * (gxn + int64_t(nx + 1) * gyn);
                if (node_fixed(support, nx, ny, nz, gxn, gyn, 0)) fix0 |= 1u << s;
                if (node_fixed(support, nx, ny, nz, gxn, gyn, 1)) fix1 |= 1u << s;
            }
        }
        gx[s] = P.x + o + kstart * plane;
        gu[s] = S ? P.u + o + kstart * plane : nullptr;
    }
    float px[PSLOT][3], pu[PSLOT][3];
    auto fetch = [&]() {   // the next plane, in order
#pragma unroll
        for (int s = 0; s < PSLOT; ++s) {
            const bool ok = (in >> s) & 1u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                px[s][c] = ok ? __ldg(gx[s] + c) : 0.0f;
                if (S) pu[s][c] = ok ? __ldg(gu[s] + c) : 0.0f;
            }
            gx[s] += plane;
            if (S) gu[s] += plane;
        }
    };
    // writes the fetched plane k into its ring slot as hi / lo, supported nodes zero (the masked
    // vectors the element matrices act on)
    auto stage = [&](int k) {
        float4* base = stg + (k & (RING - 1)) * PL + t;
        const unsigned fx = k == 0 ? fix0 : fix1;
#pragma unroll
        for (int s = 0; s < PSLOT; ++s) {
            if (!((has >> s) & 1u)) continue;
            const bool z = (fx >> s) & 1u;
            split_store(base + s * NT, base + s * NT + SLOTS, px[s], z);
            if (S) split_store(base + RING * PL + s * NT, base + RING * PL + s * NT + SLOTS, pu[s], z);
        }
    };

    // element column (lx, ly) = (lane, warp): element (X0 - 1 + lx, Y0 - 1 + ly); it is row
    // 32 (ly % 4) + lx of MMA half ly / 4, the lane this thread reads from tensor memory
    const int lx = lane, ly = wid;
    const int ex = X0 - 1 + lx, ey = Y0 - 1 + ly;
    const bool ecol = ex >= 0 && ex < nx && ey >= 0 && ey < ny;
    const bool designated = ecol && lx + 1 <= TX && ly + 1 <= TY;   // upper corner node owned here
    // owner of node (ex, ey) = local node (lx, ly), lx, ly >= 1
    const int I = ex, J = ey;
    const bool owner = lx >= 1 && ly >= 1 && I <= nx && J <= ny;
    const bool ofix0 = owner && node_fixed(support, nx, ny, nz, I, J, 0);
    const bool ofix1 = owner && node_fixed(support, nx, ny, nz, I, J, 1);
    const int orun = min(lx >> 3, SEG - 1);
    const int oslot = (ly * SEG + orun) * 9 + (lx - 8 * orun);
    const int eslot = (ly * SEG + (lx >> 3)) * 9 + (lx & 7);   // corner (0, 0) of the element
    const int64_t elayer = int64_t(nx) * ny;
    const float* wp = P.w + (ecol ? ex + int64_t(nx) * ey : 0) + kstart * elayer;
    const float* dp = S ? P.d + (ecol ? ex + int64_t(nx) * ey : 0) + kstart * elayer : nullptr;
    float4* const sq_w = sq + ly * EXT + lx;           // this row's sums (buffer 0)
    const float4* const sq_r = sq + (ly - 1) * EXT + lx;   // the row below (owners)

    const float xa = S ? P.x[P.n] : 0.0f;
    const int mode = P.mode;
    // epilogue weights, converted once and only in their mode (no FP64 work in the other modes)
    float omF = 0.0f, c0F = 0.0f, c1F = 0.0f, c2F = 0.0f;
    bool c1nz = false;
    if (mode == EPI_JACOBI) omF = float(*P.omega);
    if (mode == EPI_CHEB) {
        c0F = float(P.omega[0]);
        c1F = float(P.omega[1]);
        c2F = float(P.omega[2]);
        c1nz = c1F != 0.0f;
    }
    const bool want_dot = P.dot_slot >= 0;
    const float ks = P.kscale;
    float pdT = 0.0f, paT = 0.0f;

    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_addr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_addr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int i = t; i < 2 * (BFLOATS / 4); i += NT) sB[i] = __ldg(reinterpret_cast<const float4*>(P.B) + i);
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int p = kstart; p <= min(kstart + 2, pmax); ++p) {
        fetch();
        stage(p);
    }
    if (kstart + 3 <= pmax) fetch();
    float wn = 0.0f, dn = 0.0f;
    if (ecol && kstart < nz) {
        wn = __ldg(wp);
        if (S) dn = __ldg(dp);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // shared-memory matrix descriptors of tcgen05.mma without swizzling, as two 32-bit words: start address
    // / 16 in bits 0-13 of the low word, LBO / 16 (byte offset of the second core matrix of a K step) in
    // bits 16-29; SBO / 16 (byte offset of the next group of 8 rows) in bits 0-13 of the high word and the
    // descriptor version 1 (bit 46) in its bit 14. A: LBO 16, SBO 144; B: LBO
    // 128, SBO 1024. Offsets below are in 16-byte units.
    const uint32_t aLo = (smem_addr(stg) >> 4) | (1u << 16), bLo = (smem_addr(sB) >> 4) | (8u << 16);
    constexpr uint32_t aHi = 9u | (1u << 14), bHi = 64u | (1u << 14);
    const bool three = P.terms == 3;
    const uint32_t mbar0 = smem_addr(&mbar[0]);

    // the MMAs of MMA half h (element rows 4h .. 4h + 3) of layer k (node planes k and k + 1) into
    // accumulator buffer buf; the two halves are issued by thread 0 of warps 0 and 4, each of which
    // commits its own MMAs to the buffer's mbarrier (two arrivals per phase)
    const int my_half = t == 0 ? 0 : (t == 128 ? 1 : -1);
    auto issue = [&](int k, int buf) {
        tc_fence_after();
        const uint32_t r0 = uint32_t(k & (RING - 1)) * PL, r1 = uint32_t((k + 1) & (RING - 1)) * PL;
        const int h = my_half;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
                const uint32_t dt = tmem + uint32_t(((buf * 2 + h) * NV + v) * 32);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const uint32_t a = aLo + (s >> 1 ? r1 : r0) + uint32_t(v * RING * PL + (4 * h + (s & 1)) * SEG * 9);
                    const uint32_t b = bLo + uint32_t(s * 16);
                    tc_mma(dt, pack_desc(a, aHi), pack_desc(b, bHi), s > 0 ? 1u : 0u);
                    tc_mma(dt, pack_desc(a + SLOTS, aHi), pack_desc(b, bHi), 1u);
                    if (three) tc_mma(dt, pack_desc(a, aHi), pack_desc(b + 256, bHi), 1u);
                }
        }
        tc_commit(mbar0 + 8u * uint32_t(buf));
    };

    if (my_half >= 0) issue(kstart, 0);
    uint32_t ph = 0;   // bit b: parity of the next completion of mbar[b]
    bool ok = true;
    // top face of the previous layer (corners 4..7 become corners 0..3 of the plane above)
    float carry[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) carry[a][c] = 0.0f;
    int64_t d0 = 3 * (I + int64_t(nx + 1) * (J + int64_t(ny + 1) * kz0));
    const uint32_t lrow = tmem + (uint32_t(32 * (wid & 3)) << 16) + uint32_t((wid >> 2) * NV * 32);

    for (int k = kstart; k < kz1; ++k) {
        const int buf = (k - kstart) & 1;
        const bool layer = k < nz;
        if (my_half >= 0 && k + 1 < kz1 && k + 1 < nz) issue(k + 1, buf ^ 1);
        const float we = wn, de = dn;
        if (ecol && k + 1 < nz && k + 1 < kz1) {
            wp += elayer;
            wn = __ldg(wp);
            if (S) {
                dp += elayer;
                dn = __ldg(dp);
            }
        }
        float bot[4][3];
        if (layer) {
            if (!mbar_wait(mbar0 + 8u * uint32_t(buf), (ph >> buf) & 1u)) ok = false;
            ph ^= 1u << buf;
            __syncwarp();   // the tensor-memory loads are warp-wide (lane 0 may come from issuing)
            tc_fence_after();
            const uint32_t col = lrow + uint32_t(buf * 2 * NV * 32);
            float D[32];
            tmem_ld32(col, D);
            float yv[32];
            if (S) {
                // t_e = d_e (u_e . K_e x_e - x_alpha), u_e from the staged u (hi + lo is exact)
                const float4* u0 = stg + RING * PL + (k & (RING - 1)) * PL + eslot;
                const float4* u1 = stg + RING * PL + ((k + 1) & (RING - 1)) * PL + eslot;
                float dot = 0.0f;
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float4* up = ((a >> 2) ? u1 : u0) + ((a >> 1) & 1) * SEG * 9 + (a & 1);
                    const float4 h = up[0], l = up[SLOTS];
                    dot = fmaf(h.x + l.x, D[4 * a], dot);
                    dot = fmaf(h.y + l.y, D[4 * a + 1], dot);
                    dot = fmaf(h.z + l.z, D[4 * a + 2], dot);
                }
                const float te = de * (ks * dot - xa);
                if (designated && k + 1 >= kz0 && k + 1 < kz1) paT -= te;   // counted where its top plane is owned
                float Du[32];
                tmem_ld32(col + 32u, Du);
                const float wk = we * ks, tk = te * ks;
#pragma unroll
                for (int i = 0; i < 32; ++i) yv[i] = fmaf(wk, D[i], tk * Du[i]);
            } else {
                const float wk = we * ks;
#pragma unroll
                for (int i = 0; i < 32; ++i) yv[i] = wk * D[i];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    bot[a][c] = carry[a][c] + yv[4 * a + c];
                    carry[a][c] = yv[4 * (a + 4) + c];
                }
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    bot[a][c] = carry[a][c];
                    carry[a][c] = 0.0f;
                }
        }
        // the owner's own x on plane k: staged (masked) unless the node is supported
        float xo[3] = {0.0f, 0.0f, 0.0f};
        const bool ofixed = k == 0 ? ofix0 : ofix1;
        if (owner && k >= kz0) {
            if (ofixed) {
#pragma unroll
                for (int c = 0; c < 3; ++c) xo[c] = __ldg(P.x + d0 + c);
            } else {
                const float4* op = stg + (k & (RING - 1)) * PL + oslot;
                const float4 h = op[0], l = op[SLOTS];
                xo[0] = h.x + l.x;
                xo[1] = h.y + l.y;
                xo[2] = h.z + l.z;
            }
        }
        // corners (0, 0) and (0, 1) of this element with corners (1, 0) and (1, 1) of the element to the
        // left: the row's contributions to nodes (lx, ly) and (lx, ly + 1)
        float n0[3], n1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            n0[c] = bot[0][c] + __shfl_up_sync(0xffffffffu, bot[1][c], 1);
            n1[c] = bot[2][c] + __shfl_up_sync(0xffffffffu, bot[3][c], 1);
        }
        if (k + 3 <= pmax) {
            stage(k + 3);
            fence_async_smem();
        }
        if (k + 4 <= pmax) fetch();
        if (k >= kz0) sq_w[buf * EYT * EXT] = make_float4(n1[0], n1[1], n1[2], 0.0f);
        if (!ok) s_abort = 1;
        tc_fence_before();
        __syncthreads();
        if (s_abort) break;
        if (k < kz0) continue;
        if (owner) {
            const int gs_c = mode - EPI_GS0 - 3 * node_colour(I, J, k);   // Gauss-Seidel: the component updated
            const float4 o = sq_r[buf * EYT * EXT];
            float s3[3] = {n0[0] + o.x, n0[1] + o.y, n0[2] + o.z};
            if (ofixed) {
                s3[0] = xo[0];
                s3[1] = xo[1];
                s3[2] = xo[2];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float o3;
                if (mode == EPI_APPLY) {
                    o3 = s3[c];
                    if (want_dot) pdT += o3 * xo[c];
                } else if (mode == EPI_RESID) {
                    o3 = __ldg(P.b + d0 + c) - s3[c];
                    if (want_dot) pdT += o3 * o3;
                } else if (mode == EPI_JACOBI) {
                    const float bb = __ldg(P.b + d0 + c);
                    o3 = xo[c] + omF * ((bb - s3[c]) * __ldg(P.idiag + d0 + c));
                    if (want_dot) pdT += o3 * bb;
                } else if (mode == EPI_CHEB) {
                    const float bb = __ldg(P.b + d0 + c);
                    o3 = c0F * xo[c] + c2F * ((bb - s3[c]) * __ldg(P.idiag + d0 + c));
                    if (c1nz) o3 -= c1F * P.y[d0 + c];
                    if (want_dot) pdT += o3 * bb;
                } else {
                    const float bb = __ldg(P.b + d0 + c);
                    o3 = gs_c == c ? xo[c] + (bb - s3[c]) * __ldg(P.idiag + d0 + c) : xo[c];
                    if (want_dot) pdT += o3 * bb;
                }
                P.y[d0 + c] = o3;
            }
        }
        d0 += plane;
    }

    // tensor memory is freed before any exit; after an abandoned wait the outstanding commits are
    // waited for (bounded) first
    if (s_abort) {
        if (wid == 0) {
            mbar_wait(mbar0, ph & 1u);
            mbar_wait(mbar0 + 8u, (ph >> 1) & 1u);
        }
        __syncthreads();
    }
    if (wid == 0) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
    }
    if (s_abort) {
        if (t == 0) {
            atomicExch(&P.sc->flags[4], 1);
            P.y[0] = __int_as_float(0x7fc00000);
        }
        return;
    }

    // per-CTA partials; the last CTA finishes the dot and the alpha entry in a fixed order
    if (!want_dot && !P.with_alpha) return;
    const unsigned nblk = gridDim.x, blk = blockIdx.x;
    const double bd = tc_cta_sum<NT>(double(pdT), sred);
    const double ba = tc_cta_sum<NT>(double(paT), sred);
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
    double sd = tc_cta_sum<NT>(td, sred);
    const double sa = tc_cta_sum<NT>(ta, sred);
    if (t != 0) return;
    *P.counter = 0u;
    if (P.with_alpha) {
        const int64_t n = P.n;
        double o;
        if (mode == EPI_APPLY) {
            o = sa;
            sd += o * double(xa);
        } else if (mode == EPI_RESID) {
            o = double(P.b[n]) - sa;
            sd += o * o;
        } else if (mode == EPI_JACOBI) {
            const double bb = double(P.b[n]);
            o = double(xa) + *P.omega * ((bb - sa) * double(P.idiag[n]));
            sd += o * bb;
        } else if (mode == EPI_CHEB) {
            const double bb = double(P.b[n]);
            o = P.omega[0] * double(xa) + P.omega[2] * ((bb - sa) * double(P.idiag[n]));
            if (P.omega[1] != 0.0) o -= P.omega[1] * double(P.y[n]);
            sd += o * bb;
        } else {
            const double bb = double(P.b[n]);
            o = mode == EPI_GS0 + kGsColours ? double(xa) + (bb - sa) * double(P.idiag[n]) : double(xa);
            sd += o * bb;
        }
        P.y[n] = float(o);
    }
    if (want_dot) P.sc->red[P.dot_slot] = sd;
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
static size_t tc_smem(bool s) {
    return sizeof(float4) * (size_t(s ? 2 : 1) * tc::RING * 2 * tc::SLOTS + 2 * (tc::BFLOATS / 4) +
                             2 * tc::EYT * tc::EXT);
}

// resident CTAs per SM the kernels are built for (shared memory and 512 tensor-memory columns allow them)
constexpr int kTcMinbK = 3, kTcMinbS = 2;

static float tf32_round_host(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b += 0xFFFu + ((b >> 13) & 1u);
    b &= ~0x1FFFu;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

void tc_build(const double* Ke, std::vector<float>& B, int& terms, float& scale) {
    // the smallest D <= 4096 for which D K_e / K_e[0][0] is an integer matrix with entries below 2^11
    // (then exact in TF32)
    double s = 0.0;
    for (int D = 1; D <= 4096 && s == 0.0; ++D) {
        bool ok = true;
        for (int i = 0; i < 576 && ok; ++i) {
            const double v = D * Ke[i] / Ke[0];
            ok = std::fabs(v - std::nearbyint(v)) <= 1e-9 * D && std::fabs(v) < 2048.0;
        }
        if (ok) s = double(D) / Ke[0];
    }
    terms = s != 0.0 ? 2 : 3;
    const double sc = s != 0.0 ? s : 1.0;
    scale = float(1.0 / sc);
    B.assign(2 * tc::BFLOATS, 0.0f);
    // operand layout (K-major, no swizzle): row n (output 4 a' + c'), column k (input 4 a + c); core
    // matrices of 8 rows x 4 columns, 128 bytes each, K-adjacent ones 128 bytes apart, the next 8 rows
    // 1024 bytes further
    for (int n = 0; n < 32; ++n)
        for (int k = 0; k < 32; ++k) {
            if (n % 4 == 3 || k % 4 == 3) continue;
            const double v = sc * Ke[(3 * (n / 4) + n % 4) * 24 + 3 * (k / 4) + k % 4];
            const float hi = tf32_round_host(float(v));
            const float lo = float(v - double(hi));
            const int o = (n / 8) * 256 + (k / 4) * 32 + (n % 8) * 4 + (k % 4);
            B[o] = hi;
            B[tc::BFLOATS + o] = terms == 3 ? lo : 0.0f;
        }
    static bool attr = false;
    if (!attr) {
        PBM_CUDA(cudaFuncSetAttribute(k_tc_f32<0, kTcMinbK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(tc_smem(false))));
        PBM_CUDA(cudaFuncSetAttribute(k_tc_f32<2, kTcMinbS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(tc_smem(true))));
        attr = true;
    }
}

FusedPlan tc_plan(const Geom& G, bool op_s) {
    FusedPlan p{};
    p.var = -1;
    p.TX = tc::TX;
    p.TY = tc::TY;
    p.gx = (G.nx + 1 + p.TX - 1) / p.TX;
    p.gy = (G.ny + 1 + p.TY - 1) / p.TY;
    const int per_sm = op_s ? kTcMinbS : kTcMinbK;
    const int planes = G.nz + 1;
    const int tiles = p.gx * p.gy;
    double best = 1e300;
    p.DZ = planes;
    for (int dz = std::max(1, std::min(planes, 2)); dz <= planes; ++dz) {
        const int gz = (planes + dz - 1) / dz;
        if (dz > 1 && (planes + dz - 2) / (dz - 1) == gz && dz != planes) continue;  // same split, shorter dz
        const double waves = double((int64_t(tiles) * gz + num_sms() * per_sm - 1) / (num_sms() * per_sm));
        const double cost = waves * (dz + 1);
        if (cost < best - 1e-9) {
            best = cost;
            p.DZ = dz;
        }
    }
    p.gz = (planes + p.DZ - 1) / p.DZ;
    return p;
}

void tc_fine_f32(const FusedPlan& p, const RedSet& r, const Geom& G, const TcMatrix& tm, const float* w,
                 const float* d, const float* u, const ApplyArgs& a, cudaStream_t st) {
    const bool s = d != nullptr;
    if (!tm.B) fail(PBM_EINVAL, "tensor-core operator: element matrix not built");
    if (p.TX != tc::TX || p.TY != tc::TY) fail(PBM_EINVAL, "tensor-core operator: tile does not match the kernel");
    const int blocks = p.gx * p.gy * p.gz;
    if (2 * int64_t(blocks) > r.len) fail(PBM_EINVAL, "grid too large for the partials buffer");
    TcArgs P{};
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
    P.terms = tm.terms;
    P.kscale = tm.scale;
    P.B = tm.B;
    P.partials = r.partials;
    P.sc = r.sc;
    P.counter = r.counter;
    if (s)
        launch_pdl(k_tc_f32<2, kTcMinbS>, dim3(blocks), dim3(tc::NT), tc_smem(true), st, P);
    else
        launch_pdl(k_tc_f32<0, kTcMinbK>, dim3(blocks), dim3(tc::NT), tc_smem(false), st, P);
    PBM_LAUNCH("tensor-core FP32 fine operator");
}

}  // namespace pbm
