// Vector kernels of the Krylov solvers: casts, first Jacobi step, deterministic dot products,
// preconditioned MINRES (Paige-Saunders: Lanczos in the M^{-1} inner product, Givens QR of the
// tridiagonal matrix, three-term direction update) and the Lanczos estimate of lambda_max(D^-1 A)
// used for the Jacobi weights. Reductions are two-level and ordered (per-CTA partials in a fixed
// grid, summed by the last CTA), so every result is reproducible bit for bit. All scalars are FP64.
#include "pbm_internal.h"

namespace pbm {

constexpr int VB = 256;        // threads per vector CTA
// vector CTAs: 4 per SM, fixed for a device, so that the summation order is fixed
static int vg() { return num_sms() * 4; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// sums `v` over the CTA (valid in thread 0)
__device__ __forceinline__ double cta_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < blockDim.x / 32) ? sh[lane] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// last-CTA completion of a reduction: returns true in thread 0 of the last CTA with the total in *tot
__device__ bool finish_sum(double part, double* partials, unsigned* counter, double* tot, double* sh) {
    __shared__ bool last;
    part = cta_sum(part, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = part;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0;
    s = l2_strided_sum(partials, int(gridDim.x), threadIdx.x, blockDim.x);
    s = cta_sum(s, sh);
    if (threadIdx.x == 0) {
        *counter = 0u;
        *tot = s;
        return true;
    }
    return false;
}

// ------------------------------------------------------------------------------------------------
template <class S, class D>
__global__ void k_cast(const S* __restrict__ a, D* __restrict__ b, int64_t n) {
    pdl_wait();
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        b[i] = D(a[i]);
}

void launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, cudaStream_t st) {
    if (src32 && !dst32) launch_pdl(k_cast<float, double>, dim3(vg()), dim3(VB), 0, st, (const float*)src, (double*)dst, n);
    else if (!src32 && dst32) launch_pdl(k_cast<double, float>, dim3(vg()), dim3(VB), 0, st, (const double*)src, (float*)dst, n);
    else if (src32) launch_pdl(k_cast<float, float>, dim3(vg()), dim3(VB), 0, st, (const float*)src, (float*)dst, n);
    else launch_pdl(k_cast<double, double>, dim3(vg()), dim3(VB), 0, st, (const double*)src, (double*)dst, n);
    PBM_LAUNCH("cast");
}

void vec_zero(void* p, size_t bytes, cudaStream_t st) { PBM_CUDA(cudaMemsetAsync(p, 0, bytes, st)); }

// FP32 vectors whose base addresses are all 16-byte aligned are processed four entries per access
template <class... P>
__device__ __forceinline__ bool vec4_ok(const P*... p) {
    return ((((uintptr_t)p) & 15u) | ...) == 0;
}

// x = omega D^{-1} b (idiag = D^{-1})
template <class T>
__device__ __forceinline__ void first_jacobi_body(const T* __restrict__ b, const T* __restrict__ idiag,
                                                  const double* __restrict__ om, T* __restrict__ x, int64_t n,
                                                  unsigned blk, unsigned nblk) {
    const T w = T(*om);
    for (int64_t i = blk * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(nblk) * blockDim.x)
        x[i] = w * (b[i] * idiag[i]);
}
template <class T>
__global__ void k_first_jacobi(const T* __restrict__ b, const T* __restrict__ idiag, const double* __restrict__ om,
                               T* __restrict__ x, int64_t n) {
    pdl_wait();
    first_jacobi_body<T>(b, idiag, om, x, n, blockIdx.x, gridDim.x);
}

__global__ void k_inverse(const double* __restrict__ x, double* __restrict__ y, int64_t n, int sq) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = sq ? 1.0 / sqrt(x[i]) : 1.0 / x[i];
}
void launch_inverse(const double* x, double* y, int64_t n, cudaStream_t st) {
    k_inverse<<<vg(), VB, 0, st>>>(x, y, n, 0);
    PBM_LAUNCH("inverse");
}
void launch_inverse_sqrt(const double* x, double* y, int64_t n, cudaStream_t st) {
    k_inverse<<<vg(), VB, 0, st>>>(x, y, n, 1);
    PBM_LAUNCH("inverse sqrt");
}

void launch_scale_diag_first(pbm_grid* g, int k, bool fp32, const void* b, void* x, bool with_alpha,
                             cudaStream_t st) {
    Level& L = g->L[k];
    const int64_t n = L.g.n() + (with_alpha ? 1 : 0);
    const double* om = &g->sc->mr[16 + k];
    if (fp32) launch_pdl(k_first_jacobi<float>, dim3(vg()), dim3(VB), 0, st, (const float*)b, L.idiag32, om, (float*)x, n);
    else launch_pdl(k_first_jacobi<double>, dim3(vg()), dim3(VB), 0, st, (const double*)b, L.idiag64, om, (double*)x, n);
    PBM_LAUNCH("first jacobi");
}

template <class T>
__global__ void k_dot(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* partials, unsigned* counter,
                      double* out) {
    pdl_wait();
    __shared__ double sh[32];
    T st = T(0);   // per-thread sum in the vector type, CTA and grid sums in FP64
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        st += a[i] * b[i];
    double tot;
    if (finish_sum(double(st), partials, counter, &tot, sh)) *out = tot;
}

void launch_dot(pbm_grid* g, bool fp32, const void* a, const void* b, int64_t n, int slot, cudaStream_t st) {
    if (fp32)
        launch_pdl(k_dot<float>, dim3(vg()), dim3(VB), 0, st, (const float*)a, (const float*)b, n, g->partials, &g->sc->counter[1],
                                        &g->sc->red[slot]);
    else
        launch_pdl(k_dot<double>, dim3(vg()), dim3(VB), 0, st, (const double*)a, (const double*)b, n, g->partials, &g->sc->counter[1],
                                         &g->sc->red[slot]);
    PBM_LAUNCH("dot");
}

double read_slot(pbm_grid* g, int slot, cudaStream_t st) {
    PBM_CUDA(cudaMemcpyAsync(&g->sc_host->red[slot], &g->sc->red[slot], sizeof(double), cudaMemcpyDeviceToHost, st));
    PBM_CUDA(cudaStreamSynchronize(st));
    return g->sc_host->red[slot];
}

// ------------------------------------------------------------------------------------------------
// MINRES
//   scalar state mr[]: 0 beta_prev, 1 beta_cur, 2 c_prev, 3 s_prev, 4 c_cur, 5 s_cur, 6 eta,
//   7 eta0, 8 a_k, 9 x-step (c_new eta), 10 e_k, 11 f_k, 12 r_k, 13 status (0 ok, 1 breakdown,
//   2 r_k == 0), 14 beta_next
//   reduction slots: red[0] = A z . z, red[1] = v_next . z_next, red[2] = ||r||^2, red[3] = misc
// ------------------------------------------------------------------------------------------------
// The per-launch scalars (quotients of beta) are formed once per CTA by thread 0: FP64 division is
// a long instruction sequence on GB300, so no vector kernel divides per entry.
// Fixed-role variants: the Lanczos step writes v_next and shifts (v_prev, v_cur) <- (v_cur, v_next)
// in place; the update shifts the directions and z. Buffer roles never change between
// iterations, so every iteration is the same sequence of launches.
template <class T>
__device__ __forceinline__ void mr_lanczos2_body(const T* __restrict__ Az, T* __restrict__ v0, T* __restrict__ v1,
                                                 int64_t n, double* mr, const double* red, unsigned blk,
                                                 unsigned nblk) {
    __shared__ double cs[4];
    if (threadIdx.x == 0) {
        const double beta = mr[1], bprev = mr[0];
        const double ib = 1.0 / beta;
        const double a = red[0] * ib * ib;
        cs[0] = ib;
        cs[1] = a * ib;
        cs[2] = bprev > 0.0 ? beta / bprev : 0.0;
        cs[3] = a;
    }
    __syncthreads();
    const T c1 = T(cs[0]), c2 = T(cs[1]), c3 = T(cs[2]);   // vector arithmetic in the vector type
    auto one = [&](T az, T v0i, T& vn, T& vo) {
        const T vc = vn;
        vn = c1 * az - c2 * vc - c3 * v0i;
        vo = vc;
    };
    int64_t i0 = 0;
    if constexpr (std::is_same<T, float>::value)
    if (vec4_ok(Az, v0, v1)) {   // FP32: four entries per 16-byte access, the same arithmetic per entry
        const int64_t n4 = n / 4;
        for (int64_t q = blk * int64_t(blockDim.x) + threadIdx.x; q < n4; q += int64_t(nblk) * blockDim.x) {
            const float4 a = reinterpret_cast<const float4*>(Az)[q];
            const float4 p = reinterpret_cast<const float4*>(v0)[q];
            float4 c = reinterpret_cast<const float4*>(v1)[q], o;
            one(a.x, p.x, c.x, o.x);
            one(a.y, p.y, c.y, o.y);
            one(a.z, p.z, c.z, o.z);
            one(a.w, p.w, c.w, o.w);
            reinterpret_cast<float4*>(v1)[q] = c;
            reinterpret_cast<float4*>(v0)[q] = o;
        }
        i0 = 4 * n4;
    }
    for (int64_t i = i0 + blk * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(nblk) * blockDim.x) {
        T vn = v1[i], vo;
        one(Az[i], v0[i], vn, vo);
        v1[i] = vn;
        v0[i] = vo;
    }
    if (blk == 0 && threadIdx.x == 0) mr[8] = cs[3];
}
template <class T>
__global__ void k_mr_lanczos2(const T* __restrict__ Az, T* __restrict__ v0, T* __restrict__ v1, int64_t n,
                              double* mr, const double* red) {
    pdl_wait();
    mr_lanczos2_body<T>(Az, v0, v1, n, mr, red, blockIdx.x, gridDim.x);
}

template <class T>
__device__ __forceinline__ void mr_update2_body(T* __restrict__ zc, const T* __restrict__ zn, T* __restrict__ d1,
                                                T* __restrict__ d2, T* __restrict__ x, int64_t n, const double* mr,
                                                unsigned blk, unsigned nblk) {
    __shared__ double cs[2];
    if (threadIdx.x == 0) {
        cs[0] = 1.0 / mr[0];
        cs[1] = 1.0 / mr[12];
    }
    __syncthreads();
    const T e = T(mr[10]), f = T(mr[11]), step = T(mr[9]);
    const T ib = T(cs[0]), ir = T(cs[1]);
    // per entry: (d2, d1, x, z) <- (d1, dn, x + step dn, z_next), dn = (z / beta - e d2 - f d1) / r
    auto one = [&](T z, T d2i, T d1i, T xi, T& o2, T& o1, T& ox) {
        const T dn = (z * ib - e * d2i - f * d1i) * ir;
        o2 = d1i;
        o1 = dn;
        ox = xi + step * dn;
    };
    int64_t i0 = 0;
    if constexpr (std::is_same<T, float>::value)
    if (vec4_ok(zc, zn, d1, d2, x)) {   // FP32: four entries per 16-byte access
        const int64_t n4 = n / 4;
        for (int64_t q = blk * int64_t(blockDim.x) + threadIdx.x; q < n4; q += int64_t(nblk) * blockDim.x) {
            const float4 z = reinterpret_cast<const float4*>(zc)[q];
            const float4 a2 = reinterpret_cast<const float4*>(d2)[q];
            const float4 a1 = reinterpret_cast<const float4*>(d1)[q];
            const float4 xv = reinterpret_cast<const float4*>(x)[q];
            const float4 zz = reinterpret_cast<const float4*>(zn)[q];
            float4 o2, o1, ox;
            one(z.x, a2.x, a1.x, xv.x, o2.x, o1.x, ox.x);
            one(z.y, a2.y, a1.y, xv.y, o2.y, o1.y, ox.y);
            one(z.z, a2.z, a1.z, xv.z, o2.z, o1.z, ox.z);
            one(z.w, a2.w, a1.w, xv.w, o2.w, o1.w, ox.w);
            reinterpret_cast<float4*>(d2)[q] = o2;
            reinterpret_cast<float4*>(d1)[q] = o1;
            reinterpret_cast<float4*>(x)[q] = ox;
            reinterpret_cast<float4*>(zc)[q] = zz;
        }
        i0 = 4 * n4;
    }
    for (int64_t i = i0 + blk * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(nblk) * blockDim.x) {
        T o2, o1, ox;
        one(zc[i], d2[i], d1[i], x[i], o2, o1, ox);
        d2[i] = o2;
        d1[i] = o1;
        x[i] = ox;
        zc[i] = zn[i];
    }
}
template <class T>
__global__ void k_mr_update2(T* __restrict__ zc, const T* __restrict__ zn, T* __restrict__ d1, T* __restrict__ d2,
                             T* __restrict__ x, int64_t n, const double* mr) {
    pdl_wait();
    mr_update2_body<T>(zc, zn, d1, d2, x, n, mr, blockIdx.x, gridDim.x);
}

// dst = (double) src, red = dst . other (FP32 preconditioner output into FP64 MINRES vectors)
__global__ void k_cast_dot(const float* __restrict__ src, double* __restrict__ dst, const double* __restrict__ other,
                           int64_t n, double* partials, unsigned* counter, double* out) {
    pdl_wait();
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double v = double(src[i]);
        dst[i] = v;
        s += v * other[i];
    }
    double tot;
    if (finish_sum(s, partials, counter, &tot, sh)) *out = tot;
}

void mr_lanczos2(pbm_grid* g, bool fp32, const void* Az, void* v0, void* v1, int64_t n, cudaStream_t st) {
    if (fp32)
        launch_pdl(k_mr_lanczos2<float>, dim3(vg()), dim3(VB), 0, st, (const float*)Az, (float*)v0, (float*)v1, n, g->sc->mr, g->sc->red);
    else
        launch_pdl(k_mr_lanczos2<double>, dim3(vg()), dim3(VB), 0, st, (const double*)Az, (double*)v0, (double*)v1, n, g->sc->mr,
                                                 g->sc->red);
    PBM_LAUNCH("mr lanczos");
}
void mr_update2(pbm_grid* g, bool fp32, void* zc, const void* zn, void* d1, void* d2, void* x, int64_t n,
                cudaStream_t st) {
    if (fp32)
        launch_pdl(k_mr_update2<float>, dim3(vg()), dim3(VB), 0, st, (float*)zc, (const float*)zn, (float*)d1, (float*)d2, (float*)x, n,
                                               g->sc->mr);
    else
        launch_pdl(k_mr_update2<double>, dim3(vg()), dim3(VB), 0, st, (double*)zc, (const double*)zn, (double*)d1, (double*)d2, (double*)x,
                                                n, g->sc->mr);
    PBM_LAUNCH("mr update");
}
void cast_dot(pbm_grid* g, const float* src, double* dst, const double* other, int64_t n, int slot, cudaStream_t st) {
    launch_pdl(k_cast_dot, dim3(vg()), dim3(VB), 0, st, src, dst, other, n, g->partials, &g->sc->counter[1], &g->sc->red[slot]);
    PBM_LAUNCH("cast dot");
}

__device__ void mr_scalars_body(double* mr, const double* red) {
    const double vz = red[1];
    if (!(vz >= 0.0)) {
        mr[13] = 1.0;
        mr[9] = 0.0;
        mr[10] = mr[11] = 0.0;
        mr[12] = 1.0;
        return;
    }
    const double bnext = sqrt(vz);
    const double bcur = mr[1], a = mr[8];
    const double cp = mr[2], sp = mr[3], cc = mr[4], scur = mr[5];
    const double e = sp * bcur;
    const double gt = cp * bcur;
    const double f = cc * gt + scur * a;
    const double gk = -scur * gt + cc * a;
    const double r = hypot(gk, bnext);
    if (r == 0.0) {
        mr[13] = 2.0;
        mr[9] = 0.0;
        mr[10] = mr[11] = 0.0;
        mr[12] = 1.0;
        return;
    }
    const double cn = gk / r, sn = bnext / r;
    mr[10] = e;
    mr[11] = f;
    mr[12] = r;
    mr[9] = cn * mr[6];
    mr[6] = -sn * mr[6];
    mr[14] = bnext;
    // shift for the next iteration
    mr[0] = bcur;
    mr[1] = bnext;
    mr[2] = cc;
    mr[3] = scur;
    mr[4] = cn;
    mr[5] = sn;
}

__global__ void k_mr_scalars(double* mr, const double* red) {
    pdl_wait(); mr_scalars_body(mr, red); }

__device__ void mr_init_body(double* mr, const double* red) {
    const double vz = red[1];
    for (int i = 0; i < 16; ++i) mr[i] = 0.0;
    mr[2] = 1.0;
    mr[4] = 1.0;
    if (!(vz >= 0.0)) {
        mr[13] = 1.0;
        return;
    }
    const double b = sqrt(vz);
    mr[1] = b;
    mr[6] = b;
    mr[7] = b;
}
__global__ void k_mr_init(double* mr, const double* red) {
    pdl_wait(); mr_init_body(mr, red); }

// ---- batched vector and scalar stages of MINRES (one launch over the systems of a batch) ----
template <class T>
__global__ void k_vec_b(const VecArgs<T>* __restrict__ A, BatchMap M) {
    const int s = batch_system(M, blockIdx.x);
    if (!batch_active(M, s)) return;
    const VecArgs<T>& P = A[s];
    const unsigned blk = blockIdx.x - M.first[s], nblk = M.first[s + 1] - M.first[s];
    switch (P.op) {
        case VOP_FIRST_JACOBI: first_jacobi_body<T>(P.a, P.f, P.om, P.b, P.n, blk, nblk); break;
        case VOP_LANCZOS2: mr_lanczos2_body<T>(P.a, P.b, P.c, P.n, P.mr, P.red, blk, nblk); break;
        case VOP_UPDATE2: mr_update2_body<T>(P.b, P.a, P.c, P.d, P.e, P.n, P.mr, blk, nblk); break;
        case VOP_ZERO:
            for (int64_t i = blk * int64_t(blockDim.x) + threadIdx.x; i < P.n; i += int64_t(nblk) * blockDim.x)
                P.b[i] = T(0);
            break;
        default:  // VOP_COPY
            for (int64_t i = blk * int64_t(blockDim.x) + threadIdx.x; i < P.n; i += int64_t(nblk) * blockDim.x)
                P.b[i] = P.a[i];
            break;
    }
}
template <class T>
void launch_vec_b(const VecArgs<T>* dA, const BatchMap& M, int total_blocks, cudaStream_t st) {
    k_vec_b<T><<<total_blocks, VB, 0, st>>>(dA, M);
    PBM_LAUNCH("batched vector stage");
}
template void launch_vec_b<double>(const VecArgs<double>*, const BatchMap&, int, cudaStream_t);
template void launch_vec_b<float>(const VecArgs<float>*, const BatchMap&, int, cudaStream_t);

// one thread per system: SOP_INIT (MINRES start from red[1] = v . M^-1 v), SOP_SCALARS (Givens step)
__global__ void k_scal_b(DevScalars* const* __restrict__ sc, int nsys, int op) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    DevScalars* S = sc[s];
    if (S->flags[1] == 0) return;
    if (op == SOP_INIT) mr_init_body(S->mr, S->red);
    else mr_scalars_body(S->mr, S->red);
}
void launch_scal_b(DevScalars* const* d_sc, int nsys, int op, cudaStream_t st) {
    k_scal_b<<<(nsys + 63) / 64, 64, 0, st>>>(d_sc, nsys, op);
    PBM_LAUNCH("batched scalar stage");
}

void mr_scalars(pbm_grid* g, cudaStream_t st) {
    launch_pdl(k_mr_scalars, dim3(1), dim3(1), 0, st, g->sc->mr, g->sc->red);
    PBM_LAUNCH("mr scalars");
}
void mr_init(pbm_grid* g, cudaStream_t st) {
    launch_pdl(k_mr_init, dim3(1), dim3(1), 0, st, g->sc->mr, g->sc->red);
    PBM_LAUNCH("mr init");
}
// x64 += sign * (double) d32 (iterative refinement correction, or its removal)
__global__ void k_add_f32(double* __restrict__ x, const float* __restrict__ d, int64_t n, double sign) {
    pdl_wait();
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] += sign * double(d[i]);
}
void add_f32(double* x, const float* d, int64_t n, cudaStream_t st, double sign) {
    launch_pdl(k_add_f32, dim3(vg()), dim3(VB), 0, st, x, d, n, sign);
    PBM_LAUNCH("add f32");
}

// ------------------------------------------------------------------------------------------------
// Lanczos on D^{-1/2} A D^{-1/2}: lz_a[j], lz_b[j] (device), vectors FP64 of length n
// ------------------------------------------------------------------------------------------------
// t = s v with s = D^{-1/2} (sdiag); start vector v = 1/sqrt(n)
__global__ void k_lz_start(double* __restrict__ v, double* __restrict__ t, double* __restrict__ vprev,
                           const double* __restrict__ sdiag, int64_t n) {
    const double v0 = 1.0 / sqrt(double(n));
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        v[i] = v0;
        vprev[i] = 0.0;
        t[i] = v0 * sdiag[i];
    }
}
// w = s y - a_j v - b_{j-1} vprev (y = A s v, a_j = y . s v from the operator's fused dot); b_j = ||w||
__global__ void k_lz_b(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ vprev,
                       const double* __restrict__ sdiag, int64_t n, const double* aj, const double* bjm1,
                       double* partials, unsigned* counter, double* bj) {
    __shared__ double sh[32];
    const double a = *aj, b = bjm1 ? *bjm1 : 0.0;
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double wi = sdiag[i] * w[i] - a * v[i] - b * vprev[i];
        w[i] = wi;
        s += wi * wi;
    }
    double tot;
    if (finish_sum(s, partials, counter, &tot, sh)) *bj = sqrt(tot);
}
// vprev = v; v = w / b_j; t = s v
__global__ void k_lz_next(const double* __restrict__ w, double* __restrict__ v, double* __restrict__ vprev,
                          double* __restrict__ t, const double* __restrict__ sdiag, int64_t n, const double* bj) {
    __shared__ double ib_s;
    if (threadIdx.x == 0) {
        const double b = *bj;
        ib_s = b > 0.0 ? 1.0 / b : 0.0;
    }
    __syncthreads();
    const double ib = ib_s;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        vprev[i] = v[i];
        const double vi = w[i] * ib;
        v[i] = vi;
        t[i] = vi * sdiag[i];
    }
}

void lz_start(pbm_grid* g, double* v, double* t, double* vprev, const double* diag, int64_t n, cudaStream_t st) {
    k_lz_start<<<vg(), VB, 0, st>>>(v, t, vprev, diag, n);
    PBM_LAUNCH("lz start");
}
// j: coefficient index in sc->lz_a / lz_b; rset: reduction set of the stream (0: counter[2])
void lz_b(pbm_grid* g, double* w, const double* v, const double* vprev, const double* sdiag, int64_t n, int j0,
          int j, int rset, cudaStream_t st) {
    const RedSet r = red_set(g, rset);
    k_lz_b<<<vg(), VB, 0, st>>>(w, v, vprev, sdiag, n, &g->sc->lz_a[j0 + j], j > 0 ? &g->sc->lz_b[j0 + j - 1] : nullptr,
                              r.partials, rset == 0 ? &g->sc->counter[2] : r.counter, &g->sc->lz_b[j0 + j]);
    PBM_LAUNCH("lz b");
}
void lz_next(pbm_grid* g, const double* w, double* v, double* vprev, double* t, const double* diag, int64_t n, int j,
             cudaStream_t st) {
    k_lz_next<<<vg(), VB, 0, st>>>(w, v, vprev, t, diag, n, &g->sc->lz_b[j]);
    PBM_LAUNCH("lz next");
}

}  // namespace pbm
