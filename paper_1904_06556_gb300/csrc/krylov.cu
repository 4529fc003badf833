// Vector kernels of the Krylov solvers: casts, first Jacobi step, deterministic dot products,
// preconditioned MINRES (Paige-Saunders: Lanczos in the M^{-1} inner product, Givens QR of the
// tridiagonal matrix, three-term direction update) and the Lanczos estimate of lambda_max(D^-1 A)
// used for the Jacobi weights. Reductions are two-level and ordered (per-CTA partials in a fixed
// grid, summed by the last CTA), so every result is reproducible bit for bit. All scalars are FP64.
#include "pbm_internal.h"

namespace pbm {

constexpr int VB = 256;        // threads per vector CTA
constexpr int VG = 152 * 4;    // vector CTAs (fixed, so that the summation order is fixed)

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
    for (int i = threadIdx.x; i < int(gridDim.x); i += blockDim.x) s += ((volatile double*)partials)[i];
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
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        b[i] = D(a[i]);
}

void launch_cast(const void* src, bool src32, void* dst, bool dst32, int64_t n, cudaStream_t st) {
    if (src32 && !dst32) k_cast<float, double><<<VG, VB, 0, st>>>((const float*)src, (double*)dst, n);
    else if (!src32 && dst32) k_cast<double, float><<<VG, VB, 0, st>>>((const double*)src, (float*)dst, n);
    else if (src32) k_cast<float, float><<<VG, VB, 0, st>>>((const float*)src, (float*)dst, n);
    else k_cast<double, double><<<VG, VB, 0, st>>>((const double*)src, (double*)dst, n);
    PBM_LAUNCH("cast");
}

void vec_zero(void* p, size_t bytes, cudaStream_t st) { PBM_CUDA(cudaMemsetAsync(p, 0, bytes, st)); }

// x = omega D^{-1} b
template <class T>
__global__ void k_first_jacobi(const T* __restrict__ b, const T* __restrict__ diag, const double* __restrict__ om,
                               T* __restrict__ x, int64_t n) {
    const double w = *om;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] = T(w * double(b[i]) / double(diag[i]));
}

void launch_scale_diag_first(pbm_grid* g, int k, bool fp32, const void* b, void* x, bool with_alpha,
                             cudaStream_t st) {
    Level& L = g->L[k];
    const int64_t n = L.g.n() + (with_alpha ? 1 : 0);
    const double* om = &g->sc->mr[16 + k];
    if (fp32) k_first_jacobi<float><<<VG, VB, 0, st>>>((const float*)b, L.diag32, om, (float*)x, n);
    else k_first_jacobi<double><<<VG, VB, 0, st>>>((const double*)b, L.diag64, om, (double*)x, n);
    PBM_LAUNCH("first jacobi");
}

template <class T>
__global__ void k_dot(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* partials, unsigned* counter,
                      double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        s += double(a[i]) * double(b[i]);
    double tot;
    if (finish_sum(s, partials, counter, &tot, sh)) *out = tot;
}

void launch_dot(pbm_grid* g, bool fp32, const void* a, const void* b, int64_t n, int slot, cudaStream_t st) {
    if (fp32)
        k_dot<float><<<VG, VB, 0, st>>>((const float*)a, (const float*)b, n, g->partials, &g->sc->counter[1],
                                        &g->sc->red[slot]);
    else
        k_dot<double><<<VG, VB, 0, st>>>((const double*)a, (const double*)b, n, g->partials, &g->sc->counter[1],
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
template <class T>
__global__ void k_mr_lanczos(const T* __restrict__ Az, const T* __restrict__ vcur, T* __restrict__ vprev_next,
                             int64_t n, double* mr, const double* red) {
    const double beta = mr[1], bprev = mr[0];
    const double a = red[0] / (beta * beta);
    const double c1 = 1.0 / beta, c2 = a / beta, c3 = bprev > 0.0 ? beta / bprev : 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        vprev_next[i] = T(c1 * double(Az[i]) - c2 * double(vcur[i]) - c3 * double(vprev_next[i]));
    if (blockIdx.x == 0 && threadIdx.x == 0) mr[8] = a;
}

__global__ void k_mr_scalars(double* mr, const double* red) {
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

// d_new = (z / beta_old - e d_prev2 - f d_prev) / r  (written over d_prev2), x += step * d_new
template <class T>
__global__ void k_mr_update(const T* __restrict__ z, T* __restrict__ dprev2_new, const T* __restrict__ dprev,
                            T* __restrict__ x, int64_t n, const double* mr) {
    const double bold = mr[0];  // beta_cur of this iteration (already shifted into beta_prev)
    const double e = mr[10], f = mr[11], r = mr[12], step = mr[9];
    const double ib = 1.0 / bold, ir = 1.0 / r;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double dn = (double(z[i]) * ib - e * double(dprev2_new[i]) - f * double(dprev[i])) * ir;
        dprev2_new[i] = T(dn);
        x[i] = T(double(x[i]) + step * dn);
    }
}

__global__ void k_mr_init(double* mr, const double* red) {
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

void mr_lanczos(pbm_grid* g, bool fp32, const void* Az, const void* vcur, void* vprev_next, int64_t n, cudaStream_t st) {
    if (fp32)
        k_mr_lanczos<float><<<VG, VB, 0, st>>>((const float*)Az, (const float*)vcur, (float*)vprev_next, n, g->sc->mr,
                                               g->sc->red);
    else
        k_mr_lanczos<double><<<VG, VB, 0, st>>>((const double*)Az, (const double*)vcur, (double*)vprev_next, n,
                                                g->sc->mr, g->sc->red);
    PBM_LAUNCH("mr lanczos");
}
void mr_scalars(pbm_grid* g, cudaStream_t st) {
    k_mr_scalars<<<1, 1, 0, st>>>(g->sc->mr, g->sc->red);
    PBM_LAUNCH("mr scalars");
}
void mr_init(pbm_grid* g, cudaStream_t st) {
    k_mr_init<<<1, 1, 0, st>>>(g->sc->mr, g->sc->red);
    PBM_LAUNCH("mr init");
}
void mr_update(pbm_grid* g, bool fp32, const void* z, void* d2, const void* d1, void* x, int64_t n, cudaStream_t st) {
    if (fp32)
        k_mr_update<float><<<VG, VB, 0, st>>>((const float*)z, (float*)d2, (const float*)d1, (float*)x, n, g->sc->mr);
    else
        k_mr_update<double><<<VG, VB, 0, st>>>((const double*)z, (double*)d2, (const double*)d1, (double*)x, n,
                                               g->sc->mr);
    PBM_LAUNCH("mr update");
}

// x64 += (double) d32 (iterative refinement correction)
__global__ void k_add_f32(double* __restrict__ x, const float* __restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] += double(d[i]);
}
void add_f32(double* x, const float* d, int64_t n, cudaStream_t st) {
    k_add_f32<<<VG, VB, 0, st>>>(x, d, n);
    PBM_LAUNCH("add f32");
}

// ------------------------------------------------------------------------------------------------
// Lanczos on D^{-1/2} A D^{-1/2}: lz_a[j], lz_b[j] (device), vectors FP64 of length n
// ------------------------------------------------------------------------------------------------
// t = s v with s = 1/sqrt(D); start vector v = 1/sqrt(n)
__global__ void k_lz_start(double* __restrict__ v, double* __restrict__ t, double* __restrict__ vprev,
                           const double* __restrict__ diag, int64_t n) {
    const double v0 = 1.0 / sqrt(double(n));
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        v[i] = v0;
        vprev[i] = 0.0;
        t[i] = v0 / sqrt(diag[i]);
    }
}
// w = s w (in place), a_j = w . v
__global__ void k_lz_a(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ diag, int64_t n,
                       double* partials, unsigned* counter, double* aj) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double wi = w[i] / sqrt(diag[i]);
        w[i] = wi;
        s += wi * v[i];
    }
    double tot;
    if (finish_sum(s, partials, counter, &tot, sh)) *aj = tot;
}
// w -= a_j v + b_{j-1} vprev; b_j = ||w||
__global__ void k_lz_b(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ vprev, int64_t n,
                       const double* aj, const double* bjm1, double* partials, unsigned* counter, double* bj) {
    __shared__ double sh[32];
    const double a = *aj, b = bjm1 ? *bjm1 : 0.0;
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double wi = w[i] - a * v[i] - b * vprev[i];
        w[i] = wi;
        s += wi * wi;
    }
    double tot;
    if (finish_sum(s, partials, counter, &tot, sh)) *bj = sqrt(tot);
}
// vprev = v; v = w / b_j; t = s v
__global__ void k_lz_next(const double* __restrict__ w, double* __restrict__ v, double* __restrict__ vprev,
                          double* __restrict__ t, const double* __restrict__ diag, int64_t n, const double* bj) {
    const double b = *bj;
    const double ib = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        vprev[i] = v[i];
        const double vi = w[i] * ib;
        v[i] = vi;
        t[i] = vi / sqrt(diag[i]);
    }
}

void lz_start(pbm_grid* g, double* v, double* t, double* vprev, const double* diag, int64_t n, cudaStream_t st) {
    k_lz_start<<<VG, VB, 0, st>>>(v, t, vprev, diag, n);
    PBM_LAUNCH("lz start");
}
void lz_a(pbm_grid* g, double* w, const double* v, const double* diag, int64_t n, int j, cudaStream_t st) {
    k_lz_a<<<VG, VB, 0, st>>>(w, v, diag, n, g->partials, &g->sc->counter[2], &g->sc->lz_a[j]);
    PBM_LAUNCH("lz a");
}
void lz_b(pbm_grid* g, double* w, const double* v, const double* vprev, int64_t n, int j, cudaStream_t st) {
    k_lz_b<<<VG, VB, 0, st>>>(w, v, vprev, n, &g->sc->lz_a[j], j > 0 ? &g->sc->lz_b[j - 1] : nullptr, g->partials,
                              &g->sc->counter[2], &g->sc->lz_b[j]);
    PBM_LAUNCH("lz b");
}
void lz_next(pbm_grid* g, const double* w, double* v, double* vprev, double* t, const double* diag, int64_t n, int j,
             cudaStream_t st) {
    k_lz_next<<<VG, VB, 0, st>>>(w, v, vprev, t, diag, n, &g->sc->lz_b[j]);
    PBM_LAUNCH("lz next");
}

}  // namespace pbm
