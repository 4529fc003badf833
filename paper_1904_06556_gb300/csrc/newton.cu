// Per-element kernels of the PBM Newton step (Section 3.2, Algorithm 2).
//
// The penalty-barrier function is eq. (103.1) with tau_hat = -1/2 (pure logarithmic branch):
//   phi(t) = t + t^2/2            (t >= -1/2),   -log(-2t)/4 - 3/8   (t < -1/2)
//   phi'(t) = 1 + t                              -1/(4t)
//   phi''(t) = 1                                 1/(4t^2)
// For element i, with c_i = 1/2 u^T K_i u and s_i = (c_i - alpha + nu_lo_i - nu_up_i)/p:
//   rho'_i = rho_i phi'(s_i),  rho''_i = rho_i/p phi''(s_i),
//   mu'_lo = mu_lo phi'(-nu_lo/q_lo), mu''_lo = mu_lo/q_lo phi''(-nu_lo/q_lo) (same for up),
//   dL/dnu_lo = -rho_lo + rho' - mu'_lo,  dL/dnu_up = rho_up - rho' - mu'_up   (from eq. (aug_lagr)),
// and the elimination of (nu_lo, nu_up) from the Newton system (eq. (S)) gives per element
//   det = rho''(mu''_lo + mu''_up) + mu''_lo mu''_up,  d = rho'' mu''_lo mu''_up / det,
//   eps = rho'' (mu''_up dL/dnu_lo - mu''_lo dL/dnu_up) / det,
// so that S = [K(rho'), 0; 0, 0] + sum_i d_i [K_i u; -1][K_i u; -1]^T and
// rhs = [f - K(rho' - eps) u ; -V + sum (rho' - eps)].
#include "pbm_internal.h"

namespace pbm {

constexpr int NB = 256;
// CTAs of the element-wise kernels: 4 per SM, fixed for a device (fixed summation order)
static int ng() { return num_sms() * 4; }

__device__ __forceinline__ double phi_pb(double t) {
    return t >= -0.5 ? t + 0.5 * t * t : -0.25 * log(-2.0 * t) - 0.375;
}
__device__ __forceinline__ double dphi_pb(double t) { return t >= -0.5 ? 1.0 + t : -0.25 / t; }
__device__ __forceinline__ double ddphi_pb(double t) { return t >= -0.5 ? 1.0 : 0.25 / (t * t); }

// ordered multi-value reduction over a fixed grid; the last CTA writes out[0..NV)
template <int NV>
__device__ void finish_multi(double (&v)[NV], double* partials, unsigned* counter, double* out) {
    __shared__ double sh[NV][NB / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < NB / 32; ++w) s += sh[q][w];
            partials[q * gridDim.x + blockIdx.x] = s;
        }
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int b = 0; b < int(gridDim.x); ++b) s += ((volatile double*)partials)[threadIdx.x * gridDim.x + b];
        out[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
}

// coefficient kernel. c = per-element u^T K_e u (already computed). Outputs:
//   w = rho', d, eps, aux = rho' - eps, coef[0..4][m] = rho'', mu''_lo, mu''_up, gl, gu.
// sums: 0 sum d, 1 sum rho', 2 sum (rho' - eps), 3 ||gl||^2, 4 #bad
__global__ void k_coeffs(int64_t m, const double* __restrict__ c2, const double* __restrict__ rho,
                         const double* __restrict__ mul, const double* __restrict__ muu, const double* __restrict__ nul,
                         const double* __restrict__ nuu, double alpha, double p, double ql, double qu, double rho_lo,
                         double rho_up, double* __restrict__ w, double* __restrict__ d, double* __restrict__ eps,
                         double* __restrict__ aux, double* __restrict__ coef, double* partials, unsigned* counter,
                         double* out) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double ce = 0.5 * c2[e];
        const double s = (ce - alpha + nul[e] - nuu[e]) / p;
        const double r1 = rho[e] * dphi_pb(s);
        const double r2 = rho[e] / p * ddphi_pb(s);
        const double tl = -nul[e] / ql, tu = -nuu[e] / qu;
        const double ml1 = mul[e] * dphi_pb(tl), ml2 = mul[e] / ql * ddphi_pb(tl);
        const double mu1 = muu[e] * dphi_pb(tu), mu2 = muu[e] / qu * ddphi_pb(tu);
        const double gl = -rho_lo + r1 - ml1;
        const double gu = rho_up - r1 - mu1;
        const double det = r2 * (ml2 + mu2) + ml2 * mu2;
        const double de = r2 * ml2 * mu2 / det;
        const double ep = r2 * (mu2 * gl - ml2 * gu) / det;
        w[e] = r1;
        d[e] = de;
        eps[e] = ep;
        aux[e] = r1 - ep;
        coef[e] = r2;
        coef[m + e] = ml2;
        coef[2 * m + e] = mu2;
        coef[3 * m + e] = gl;
        coef[4 * m + e] = gu;
        acc[0] += de;
        acc[1] += r1;
        acc[2] += r1 - ep;
        acc[3] += gl * gl;
        const bool ok = isfinite(de) && isfinite(ep) && r1 > 0.0 && r2 > 0.0 && de > 0.0;
        acc[4] += ok ? 0.0 : 1.0;
    }
    finish_multi<5>(acc, partials, counter, out);
}

void launch_coeffs(pbm_grid* g, const pbm_state* s, const double* c2, double* coef, cudaStream_t st) {
    const int64_t m = g->L[0].g.m();
    k_coeffs<<<ng(), NB, 0, st>>>(m, c2, s->rho_dev, s->mu_lo_dev, s->mu_up_dev, s->nu_lo_dev, s->nu_up_dev, s->alpha,
                                s->p, s->q_lo, s->q_up, s->rho_lo, s->rho_up, g->w64, g->d64, g->eps64, g->wr64, coef,
                                g->partials, &g->sc->counter[3], &g->sc->red[8]);
    PBM_LAUNCH("coeffs");
}

// set one vector entry from a device scalar: y[i] = a * src + b
__global__ void k_set_entry(double* y, int64_t i, const double* src, double a, double b) { y[i] = a * (*src) + b; }
void set_entry(double* y, int64_t i, const double* src, double a, double b, cudaStream_t st) {
    k_set_entry<<<1, 1, 0, st>>>(y, i, src, a, b);
    PBM_LAUNCH("set entry");
}

// finite and >= 0 check: out[0] = #bad
__global__ void k_check_nonneg(const double* __restrict__ v, int64_t n, double* partials, unsigned* counter,
                               double* out) {
    double acc[1] = {0.0};
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        acc[0] += (isfinite(v[i]) && v[i] >= 0.0) ? 0.0 : 1.0;
    finish_multi<1>(acc, partials, counter, out);
}
void launch_check_nonneg(pbm_grid* g, const double* v, int64_t n, int slot, cudaStream_t st) {
    k_check_nonneg<<<ng(), NB, 0, st>>>(v, n, g->partials, &g->sc->counter[3], &g->sc->red[slot]);
    PBM_LAUNCH("check");
}

// masked copy: y = x with supported dofs zeroed (fine level)
__global__ void k_mask_copy(int nx, int ny, int nz, int support, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t nn = int64_t(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t nd = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; nd < nn; nd += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(nd % (nx + 1)), j = int((nd / (nx + 1)) % (ny + 1)), k = int(nd / (int64_t(nx + 1) * (ny + 1)));
        const bool fx = node_fixed(support, nx, ny, nz, i, j, k);
        for (int c = 0; c < 3; ++c) y[3 * nd + c] = fx ? 0.0 : x[3 * nd + c];
    }
}
void launch_mask_copy(pbm_grid* g, const double* x, double* y, cudaStream_t st) {
    const Geom& G = g->L[0].g;
    k_mask_copy<<<ng(), NB, 0, st>>>(G.nx, G.ny, G.nz, G.support, x, y);
    PBM_LAUNCH("mask copy");
}

// eq. (deltanu): dnu = -B^{-1} (grad_nu L + rho'' (w . du - dalpha) [1; -1]); bq = w_e . du_e
__global__ void k_delta_nu(int64_t m, const double* __restrict__ bq, const double* __restrict__ coef,
                           const double* __restrict__ dz_alpha, double* __restrict__ dl, double* __restrict__ du) {
    const double da = *dz_alpha;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double r2 = coef[e], ml2 = coef[m + e], mu2 = coef[2 * m + e], gl = coef[3 * m + e], gu = coef[4 * m + e];
        const double proj = bq[e] - da;
        const double rl = gl + r2 * proj, ru = gu - r2 * proj;
        const double a11 = r2 + ml2, a22 = r2 + mu2, a12 = -r2;
        const double det = a11 * a22 - a12 * a12;
        dl[e] = -(a22 * rl - a12 * ru) / det;
        du[e] = -(-a12 * rl + a11 * ru) / det;
    }
}
void launch_delta_nu(pbm_grid* g, const double* bq, const double* coef, const double* dz_alpha, double* dl, double* du,
                     cudaStream_t st) {
    k_delta_nu<<<ng(), NB, 0, st>>>(g->L[0].g.m(), bq, coef, dz_alpha, dl, du);
    PBM_LAUNCH("delta nu");
}

// penalty sums of the augmented Lagrangian at step kappa along (du, dnu):
//   out[0] = sum rho p phi(s(kappa)) + mu_lo q_lo phi(-(nu_lo + k dl)/q_lo) + mu_up q_up phi(..)
//   out[1] = sum (nu_lo + k dl), out[2] = sum (nu_up + k dup), out[3] = #infeasible (log branch domain)
// with c(kappa) = c0 + kappa b + kappa^2 q / 2 from the per-element forms c0 = u^T K u / 2,
// b = u^T K du, q = du^T K du.
__global__ void k_lagr_terms(int64_t m, double kappa, const double* __restrict__ c2u, const double* __restrict__ bq,
                             const double* __restrict__ qq, const double* __restrict__ rho,
                             const double* __restrict__ mul, const double* __restrict__ muu,
                             const double* __restrict__ nul, const double* __restrict__ nuu,
                             const double* __restrict__ dl, const double* __restrict__ dup, double alpha_k, double p,
                             double ql, double qu, double* partials, unsigned* counter, double* out) {
    double acc[4] = {0, 0, 0, 0};
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double ce = 0.5 * c2u[e] + kappa * bq[e] + 0.5 * kappa * kappa * qq[e];
        const double nl = nul[e] + kappa * dl[e], nu = nuu[e] + kappa * dup[e];
        const double s = (ce - alpha_k + nl - nu) / p;
        const double v = rho[e] * p * phi_pb(s) + mul[e] * ql * phi_pb(-nl / ql) + muu[e] * qu * phi_pb(-nu / qu);
        acc[0] += v;
        acc[1] += nl;
        acc[2] += nu;
        acc[3] += isfinite(v) ? 0.0 : 1.0;
    }
    finish_multi<4>(acc, partials, counter, out);
}
void launch_lagr_terms(pbm_grid* g, double kappa, const double* c2u, const double* bq, const double* qq,
                       const pbm_state* s, const double* dl, const double* dup, double alpha_k, int slot,
                       cudaStream_t st) {
    k_lagr_terms<<<ng(), NB, 0, st>>>(g->L[0].g.m(), kappa, c2u, bq, qq, s->rho_dev, s->mu_lo_dev, s->mu_up_dev,
                                    s->nu_lo_dev, s->nu_up_dev, dl, dup, alpha_k, s->p, s->q_lo, s->q_up, g->partials,
                                    &g->sc->counter[3], &g->sc->red[slot]);
    PBM_LAUNCH("lagr terms");
}

// y += kappa x (n)
__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double kappa, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += kappa * x[i];
}
void launch_axpy(double* y, const double* x, double kappa, int64_t n, cudaStream_t st) {
    k_axpy<<<ng(), NB, 0, st>>>(y, x, kappa, n);
    PBM_LAUNCH("axpy");
}

// per-element c = u^T K_e u / 2 (compliance) from the bilinear form
__global__ void k_scale(const double* __restrict__ a, double* __restrict__ b, double s, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        b[i] = s * a[i];
}
void launch_scale(const double* a, double* b, double s, int64_t n, cudaStream_t st) {
    k_scale<<<ng(), NB, 0, st>>>(a, b, s, n);
    PBM_LAUNCH("scale");
}

// Algorithm 1 multiplier update with the safeguard beta x <= x+ <= x / beta (ibeta = 1 / beta):
//   rho+ = rho phi'(s), mu_lo+ = mu_lo phi'(-nu_lo / q_lo), mu_up+ = mu_up phi'(-nu_up / q_up),
// s = (c - alpha + nu_lo - nu_up) / p, c = u^T K_e u / 2 (c2 holds u^T K_e u).
__global__ void k_mult_update(int64_t m, const double* __restrict__ c2, double* __restrict__ rho,
                              double* __restrict__ mul, double* __restrict__ muu, const double* __restrict__ nul,
                              const double* __restrict__ nuu, double alpha, double p, double ql, double qu,
                              double beta, double ibeta, int only_rho) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double s = (0.5 * c2[e] - alpha + nul[e] - nuu[e]) / p;
        const double r = rho[e];
        rho[e] = fmin(fmax(r * dphi_pb(s), beta * r), r * ibeta);
        if (only_rho) continue;
        const double a = mul[e], b = muu[e];
        mul[e] = fmin(fmax(a * dphi_pb(-nul[e] / ql), beta * a), a * ibeta);
        muu[e] = fmin(fmax(b * dphi_pb(-nuu[e] / qu), beta * b), b * ibeta);
    }
}
void launch_mult_update(pbm_grid* g, const double* c2, pbm_state* s, double beta, bool only_rho, cudaStream_t st) {
    k_mult_update<<<ng(), NB, 0, st>>>(g->L[0].g.m(), c2, s->rho_dev, s->mu_lo_dev, s->mu_up_dev, s->nu_lo_dev,
                                     s->nu_up_dev, s->alpha, s->p, s->q_lo, s->q_up, beta, 1.0 / beta,
                                     only_rho ? 1 : 0);
    PBM_LAUNCH("multiplier update");
}

// sums of the duality gap (eq. gap) and the dual objective: out[0] = sum min(rho_lo a, rho_up a),
// a = alpha - c_e; out[1] = sum nu_lo; out[2] = sum nu_up; out[3] = sum rho
__global__ void k_gap_sums(int64_t m, const double* __restrict__ c2, double alpha, double rho_lo, double rho_up,
                           const double* __restrict__ nul, const double* __restrict__ nuu,
                           const double* __restrict__ rho, double* partials, unsigned* counter, double* out) {
    double acc[4] = {0, 0, 0, 0};
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double a = alpha - 0.5 * c2[e];
        acc[0] += fmin(rho_lo * a, rho_up * a);
        acc[1] += nul[e];
        acc[2] += nuu[e];
        acc[3] += rho[e];
    }
    finish_multi<4>(acc, partials, counter, out);
}
void launch_gap_sums(pbm_grid* g, const double* c2, const pbm_state* s, int slot, cudaStream_t st) {
    k_gap_sums<<<ng(), NB, 0, st>>>(g->L[0].g.m(), c2, s->alpha, s->rho_lo, s->rho_up, s->nu_lo_dev, s->nu_up_dev,
                                  s->rho_dev, g->partials, &g->sc->counter[3], &g->sc->red[slot]);
    PBM_LAUNCH("gap sums");
}

}  // namespace pbm

// ------------------------------------------------------------------------------------------------
// Interior-point Newton system (Section 4.1). With c2 = u_e^T K_e u_e per element:
//   res_3 = c2/2 + alpha + nu_lo - nu_up,  res_4 = nu_lo (rho - rho_lo) - r,  res_5 = nu_up (rho_up - rho) - s,
//   d = 1 / (nu_lo / (rho - rho_lo) + nu_up / (rho_up - rho)),
//   c = res_3 - res_4 / (rho - rho_lo) + res_5 / (rho_up - rho)        (from J dz = -res, eq. (gradres)),
// so that S_IP = [K(rho), 0; 0, 0] + sum_i d_i [K_i u; 1][K_i u; 1]^T (eq. (S_IP)) and the right-hand side is
// [f - K(rho + d c) u ; V - sum(rho + d c)].
// ------------------------------------------------------------------------------------------------
namespace pbm {

// outputs: w = rho, d, wr = rho + d c, coef rows c, res_3, res_4, res_5, nu_lo - nu_up;
// sums: 0 sum d, 1 sum (rho + d c), 2 #elements not strictly feasible or not finite
__global__ void k_ip_coeffs(int64_t m, const double* __restrict__ c2, const double* __restrict__ rho,
                            const double* __restrict__ nul, const double* __restrict__ nuu, double alpha, double rho_lo,
                            double rho_up, double r, double s, double* __restrict__ w, double* __restrict__ d,
                            double* __restrict__ wr, double* __restrict__ coef, double* partials, unsigned* counter,
                            double* out) {
    double acc[3] = {0, 0, 0};
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double re = rho[e], nl = nul[e], nu = nuu[e];
        const double gl = re - rho_lo, gu = rho_up - re;
        const double r3 = 0.5 * c2[e] + alpha + nl - nu;
        const double r4 = nl * gl - r;
        const double r5 = nu * gu - s;
        const double de = 1.0 / (nl / gl + nu / gu);
        const double ce = r3 - r4 / gl + r5 / gu;
        w[e] = re;
        d[e] = de;
        wr[e] = re + de * ce;
        coef[e] = ce;
        coef[m + e] = r3;
        coef[2 * m + e] = r4;
        coef[3 * m + e] = r5;
        coef[4 * m + e] = nl - nu;
        acc[0] += de;
        acc[1] += re + de * ce;
        const bool ok = gl > 0.0 && gu > 0.0 && nl > 0.0 && nu > 0.0 && isfinite(de) && isfinite(ce) && de > 0.0;
        acc[2] += ok ? 0.0 : 1.0;
    }
    finish_multi<3>(acc, partials, counter, out);
}

void launch_ip_coeffs(pbm_grid* g, const pbm_ip_state* s, const double* c2, double* coef, cudaStream_t st) {
    const int64_t m = g->L[0].g.m();
    k_ip_coeffs<<<ng(), NB, 0, st>>>(m, c2, s->rho_dev, s->nu_lo_dev, s->nu_up_dev, s->alpha, s->rho_lo, s->rho_up, s->r,
                                   s->s, g->w64, g->d64, g->wr64, coef, g->partials, &g->sc->counter[3],
                                   &g->sc->red[8]);
    PBM_LAUNCH("ip coeffs");
}

// increments from the reduced solution: wdu = u_e^T K_e du_e, da = dz[n];
//   drho = d (wdu + da + c),
//   dnu_up = ((rho - rho_lo)(wdu + da + res_3) - (nu_lo - nu_up) drho - res_4 - res_5) / (rho_up - rho_lo),
//   dnu_lo = dnu_up - wdu - da - res_3
__global__ void k_ip_recover(int64_t m, const double* __restrict__ wdu, const double* __restrict__ da_p,
                             const double* __restrict__ rho, const double* __restrict__ d,
                             const double* __restrict__ coef, double rho_lo, double rho_up, double* __restrict__ drho,
                             double* __restrict__ dnl, double* __restrict__ dnu) {
    const double da = *da_p;
    const double inv = 1.0 / (rho_up - rho_lo);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const double ce = coef[e], r3 = coef[m + e], r4 = coef[2 * m + e], r5 = coef[3 * m + e];
        const double ndiff = coef[4 * m + e];
        const double q = wdu[e] + da;
        const double dr = d[e] * (q + ce);
        const double du_ = ((rho[e] - rho_lo) * (q + r3) - ndiff * dr - r4 - r5) * inv;
        drho[e] = dr;
        dnu[e] = du_;
        dnl[e] = du_ - q - r3;
    }
}

void launch_ip_recover(pbm_grid* g, const double* wdu, const double* da, const double* coef, double rho_lo,
                       double rho_up, double* drho, double* dnl, double* dnu, cudaStream_t st) {
    const int64_t m = g->L[0].g.m();
    k_ip_recover<<<ng(), NB, 0, st>>>(m, wdu, da, g->w64, g->d64, coef, rho_lo, rho_up, drho, dnl, dnu);
    PBM_LAUNCH("ip recover");
}

}  // namespace pbm

// ------------------------------------------------------------------------------------------------
// Damped optimality-criteria step (Algorithm DOC, Section 4.2): with e_i = u^T K_i u the trial density
// of a volume multiplier alpha is rho_i^+ = min(max(w_i / alpha, rho_lo), rho_up), w_i = rho_i e_i^q.
// The bisection state lives on the device (ctl[0] lo, ctl[1] hi, ctl[2] alpha of the last trial,
// ctl[3] trials, ctl[4] done), so the trials run as consecutive launches without host round trips.
// ------------------------------------------------------------------------------------------------
namespace pbm {

__global__ void k_doc_weights(int64_t m, const double* __restrict__ rho, const double* __restrict__ e, double q,
                              double* __restrict__ w, double* ctl, double alpha_hi) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
        w[i] = rho[i] * pow(e[i], q);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl[0] = 0.0;
        ctl[1] = alpha_hi;
        ctl[2] = 0.0;
        ctl[3] = 0.0;
        ctl[4] = 0.0;
    }
}

// one trial: if the interval is still wide, alpha = its midpoint, the sum of the trial densities, and the last
// CTA moves one end of the interval (every CTA reads the interval before any CTA can reach the update)
__global__ void k_doc_trial(int64_t m, const double* __restrict__ w, double V, double rho_lo, double rho_up,
                            double tau, double* ctl, double* partials, unsigned* counter) {
    __shared__ double sh[NB / 32];
    __shared__ bool last;
    const double lo = ctl[0], hi = ctl[1];
    if (ctl[4] != 0.0) return;
    if ((hi - lo) / (hi + lo) <= tau) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl[4] = 1.0;
        return;
    }
    const double alpha = 0.5 * (hi + lo);
    double s = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
        s += fmin(fmax(w[i] / alpha, rho_lo), rho_up);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < NB / 32; ++k) b += sh[k];
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double tot = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) tot += ((volatile double*)partials)[k];
    ctl[2] = alpha;
    ctl[3] += 1.0;
    if (tot > V) ctl[0] = alpha;
    else ctl[1] = alpha;
    *counter = 0u;
}

// rho^+ from the last trial's alpha (rho unchanged if no trial ran); out[0] = ||rho^+ - rho||_inf
__global__ void k_doc_update(int64_t m, const double* __restrict__ w, const double* ctl, double rho_lo,
                             double rho_up, const double* __restrict__ rho, double* __restrict__ rho_new,
                             double* partials, unsigned* counter, double* out) {
    __shared__ double sh[NB / 32];
    __shared__ bool last;
    const bool none = ctl[3] == 0.0;
    const double alpha = ctl[2];
    double mx = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const double r = none ? rho[i] : fmin(fmax(w[i] / alpha, rho_lo), rho_up);
        mx = fmax(mx, fabs(r - rho[i]));
        rho_new[i] = r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < NB / 32; ++k) b = fmax(b, sh[k]);
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double tot = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) tot = fmax(tot, ((volatile double*)partials)[k]);
    *out = tot;
    *counter = 0u;
}

void launch_doc(pbm_grid* g, const double* e, double* rho_inout, double V, double rho_lo, double rho_up, double q,
                double tau, double* w, cudaStream_t st) {
    const int64_t m = g->L[0].g.m();
    double* ctl = &g->sc->ctl[0];   // reused: the MINRES loop is not running
    k_doc_weights<<<ng(), NB, 0, st>>>(m, g->rho, e, q, w, ctl, 1e4);
    PBM_LAUNCH("doc weights");
    // trials in batches; the host looks at the done flag after each batch
    for (int batch = 0; batch < 8; ++batch) {
        for (int t = 0; t < 16; ++t) {
            k_doc_trial<<<ng(), NB, 0, st>>>(m, w, V, rho_lo, rho_up, tau, ctl, g->partials, &g->sc->counter[3]);
            PBM_LAUNCH("doc trial");
        }
        PBM_CUDA(cudaMemcpyAsync(&g->sc_host->ctl[0], ctl, sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
        PBM_CUDA(cudaStreamSynchronize(st));
        if (g->sc_host->ctl[4] != 0.0) break;
    }
    if (g->sc_host->ctl[4] == 0.0) fail(PBM_ENOTCONV, "DOC bisection did not close its interval in 128 trials");
    k_doc_update<<<ng(), NB, 0, st>>>(m, w, ctl, rho_lo, rho_up, g->rho, rho_inout, g->partials, &g->sc->counter[3],
                                    &g->sc->red[12]);
    PBM_LAUNCH("doc update");
}

}  // namespace pbm
