// NCL outer loop (Section IV-A, eq. nclsubpb) and interior-point inner loop
// (Section IV-B) with device-resident iterates.
//
// Every vector operation runs on the GPU; each iteration brings back only a
// handful of per-CTA partial reductions (summed on the host in a fixed
// order, so runs are repeatable).  The control logic follows the published
// algorithms the paper builds on and is the same as the CPU oracle's:
//  * outer: accept lam_n += rho r, nu0_n += rho t when max(|r|,|t|) <= eta
//    (then eta, omega /= 10), else rho *= 10; infeasible once rho > rho_max;
//  * inner (Waechter & Biegler 2006): monotone Fiacco-McCormick barrier
//    update, inertia correction with delta_w, fraction-to-boundary, filter
//    line search, bound-multiplier safeguard;
//  * mixed precision: FP32 block factors with FP64 refinement; when the
//    refinement stalls the step is redone with FP64 factors, and the rest of
//    the solve stays in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

#include "handle.h"

namespace scopf {

namespace {

constexpr int kT = 256;
constexpr int kB = 296;  // CTAs of the reduction kernels (2 per SM)

struct Dev {
    const double *wl, *wu;
    const int64_t *c1, *c2;
    int64_t n, m, p;
};

// ---- per-CTA partial reductions ---------------------------------------
__device__ double block_reduce(double v, int op, double *sh) {
    // op: 0 max, 1 min, 2 sum
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            double a = sh[threadIdx.x], b = sh[threadIdx.x + s];
            sh[threadIdx.x] = op == 0 ? fmax(a, b) : (op == 1 ? fmin(a, b) : a + b);
        }
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// w-part: [max|gwz|, min sl*zl, max sl*zl, min su*zu, max su*zu, sum|zl|, sum|zu|]
__global__ void k_red_w(Dev D, const double *w, const double *gw, const double *zl,
                        const double *zu, double *part) {
    __shared__ double sh[kT];
    double a0 = 0, a1 = INFINITY, a2 = -INFINITY, a3 = INFINITY, a4 = -INFINITY, a5 = 0, a6 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double g = gw[i];
        const double l = D.wl[i], u = D.wu[i], x = w[i];
        if (l > -INFINITY) {
            g -= zl[i];
            const double c = (x - l) * zl[i];
            a1 = fmin(a1, c);
            a2 = fmax(a2, c);
            a5 += fabs(zl[i]);
        }
        if (u < INFINITY) {
            g += zu[i];
            const double c = (u - x) * zu[i];
            a3 = fmin(a3, c);
            a4 = fmax(a4, c);
            a6 += fabs(zu[i]);
        }
        a0 = fmax(a0, fabs(g));
    }
    double *o = part + (int64_t)blockIdx.x * 7;
    double r;
    r = block_reduce(a0, 0, sh); if (threadIdx.x == 0) o[0] = r;
    r = block_reduce(a1, 1, sh); if (threadIdx.x == 0) o[1] = r;
    r = block_reduce(a2, 0, sh); if (threadIdx.x == 0) o[2] = r;
    r = block_reduce(a3, 1, sh); if (threadIdx.x == 0) o[3] = r;
    r = block_reduce(a4, 0, sh); if (threadIdx.x == 0) o[4] = r;
    r = block_reduce(a5, 2, sh); if (threadIdx.x == 0) o[5] = r;
    r = block_reduce(a6, 2, sh); if (threadIdx.x == 0) o[6] = r;
}

// m-part: [max|gr|, max|c-r|, sum|c-r|, sum|lam|, max|r|]
__global__ void k_red_m(Dev D, const double *c, const double *r, const double *lam,
                        const double *lam_n, DScalar rho_, double *part) {
    __shared__ double sh[kT];
    const double rho = rho_.get();
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D.m;
         i += (int64_t)gridDim.x * blockDim.x) {
        a0 = fmax(a0, fabs(lam_n[i] + rho * r[i] - lam[i]));
        const double pc = fabs(c[i] - r[i]);
        a1 = fmax(a1, pc);
        a2 += pc;
        a3 += fabs(lam[i]);
        a4 = fmax(a4, fabs(r[i]));
    }
    double *o = part + (int64_t)blockIdx.x * 5;
    double v;
    v = block_reduce(a0, 0, sh); if (threadIdx.x == 0) o[0] = v;
    v = block_reduce(a1, 0, sh); if (threadIdx.x == 0) o[1] = v;
    v = block_reduce(a2, 2, sh); if (threadIdx.x == 0) o[2] = v;
    v = block_reduce(a3, 2, sh); if (threadIdx.x == 0) o[3] = v;
    v = block_reduce(a4, 0, sh); if (threadIdx.x == 0) o[4] = v;
}

// p-part: [max|gt|, max|gs|, max|py|, sum|py|, min s zs, max s zs, sum|yc|, sum|zs|, max|t|]
__global__ void k_red_p(Dev D, const double *w, const double *t, const double *s,
                        const double *yc, const double *zs, const double *nu0_n, DScalar rho_,
                        double *part) {
    __shared__ double sh[kT];
    const double rho = rho_.get();
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = INFINITY, a5 = -INFINITY, a6 = 0, a7 = 0, a8 = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < D.p;
         q += (int64_t)gridDim.x * blockDim.x) {
        a0 = fmax(a0, fabs(nu0_n[q] + rho * t[q] - yc[q]));
        a1 = fmax(a1, fabs(yc[q] - zs[q]));
        const double py = fabs(w[D.c1[q]] * w[D.c2[q]] - t[q] + s[q]);
        a2 = fmax(a2, py);
        a3 += py;
        const double cz = s[q] * zs[q];
        a4 = fmin(a4, cz);
        a5 = fmax(a5, cz);
        a6 += fabs(yc[q]);
        a7 += fabs(zs[q]);
        a8 = fmax(a8, fabs(t[q]));
    }
    double *o = part + (int64_t)blockIdx.x * 9;
    double v;
    v = block_reduce(a0, 0, sh); if (threadIdx.x == 0) o[0] = v;
    v = block_reduce(a1, 0, sh); if (threadIdx.x == 0) o[1] = v;
    v = block_reduce(a2, 0, sh); if (threadIdx.x == 0) o[2] = v;
    v = block_reduce(a3, 2, sh); if (threadIdx.x == 0) o[3] = v;
    v = block_reduce(a4, 1, sh); if (threadIdx.x == 0) o[4] = v;
    v = block_reduce(a5, 0, sh); if (threadIdx.x == 0) o[5] = v;
    v = block_reduce(a6, 2, sh); if (threadIdx.x == 0) o[6] = v;
    v = block_reduce(a7, 2, sh); if (threadIdx.x == 0) o[7] = v;
    v = block_reduce(a8, 0, sh); if (threadIdx.x == 0) o[8] = v;
}

// barrier objective pieces at a state: [sum ln(slacks of w), sum ln s, lam_n'r + rho/2 r'r,
// nu0_n't + rho/2 t't, number of nonpositive slacks]
__global__ void k_barrier(Dev D, const double *w, const double *r, const double *t,
                          const double *s, const double *lam_n, const double *nu0_n, DScalar rho_,
                          double *part) {
    __shared__ double sh[kT];
    const double rho = rho_.get();
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    const int64_t tot = D.n + D.m + D.p;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < D.n) {
            const double l = D.wl[i], u = D.wu[i], x = w[i];
            if (l > -INFINITY) {
                if (x - l > 0) a0 += log(x - l); else a4 += 1;
            }
            if (u < INFINITY) {
                if (u - x > 0) a0 += log(u - x); else a4 += 1;
            }
        } else if (i < D.n + D.m) {
            const int64_t j = i - D.n;
            a2 += lam_n[j] * r[j] + 0.5 * rho * r[j] * r[j];
        } else {
            const int64_t q = i - D.n - D.m;
            if (s[q] > 0) a1 += log(s[q]); else a4 += 1;
            a3 += nu0_n[q] * t[q] + 0.5 * rho * t[q] * t[q];
        }
    }
    double *o = part + (int64_t)blockIdx.x * 5;
    double v;
    v = block_reduce(a0, 2, sh); if (threadIdx.x == 0) o[0] = v;
    v = block_reduce(a1, 2, sh); if (threadIdx.x == 0) o[1] = v;
    v = block_reduce(a2, 2, sh); if (threadIdx.x == 0) o[2] = v;
    v = block_reduce(a3, 2, sh); if (threadIdx.x == 0) o[3] = v;
    v = block_reduce(a4, 2, sh); if (threadIdx.x == 0) o[4] = v;
}

// directional derivative of the barrier objective:
// [g'dw, -mu sum dw/sl + mu sum dw/su, (lam_n + rho r)'dr, (nu0_n + rho t)'dt, -mu sum ds/s]
__global__ void k_dirderiv(Dev D, const double *w, const double *g, const double *r,
                           const double *t, const double *s, const double *lam_n,
                           const double *nu0_n, DScalar rho_, DScalar mu_, const double *dw,
                           const double *dr, const double *dt, const double *ds, double *part) {
    __shared__ double sh[kT];
    const double rho = rho_.get(), mu = mu_.get();
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    const int64_t tot = D.n + D.m + D.p;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < D.n) {
            a0 += g[i] * dw[i];
            const double l = D.wl[i], u = D.wu[i], x = w[i];
            if (l > -INFINITY) a1 -= mu * dw[i] / (x - l);
            if (u < INFINITY) a1 += mu * dw[i] / (u - x);
        } else if (i < D.n + D.m) {
            const int64_t j = i - D.n;
            a2 += (lam_n[j] + rho * r[j]) * dr[j];
        } else {
            const int64_t q = i - D.n - D.m;
            a3 += (nu0_n[q] + rho * t[q]) * dt[q];
            a4 -= mu * ds[q] / s[q];
        }
    }
    double *o = part + (int64_t)blockIdx.x * 5;
    double v;
    v = block_reduce(a0, 2, sh); if (threadIdx.x == 0) o[0] = v;
    v = block_reduce(a1, 2, sh); if (threadIdx.x == 0) o[1] = v;
    v = block_reduce(a2, 2, sh); if (threadIdx.x == 0) o[2] = v;
    v = block_reduce(a3, 2, sh); if (threadIdx.x == 0) o[3] = v;
    v = block_reduce(a4, 2, sh); if (threadIdx.x == 0) o[4] = v;
}

// fraction to boundary: [alpha_primal, alpha_dual]
__global__ void k_ftb(Dev D, const double *w, const double *s, const double *zl,
                      const double *zu, const double *zs, const double *dw, const double *ds,
                      const double *dzl, const double *dzu, const double *dzs, DScalar tau_,
                      double *part) {
    __shared__ double sh[kT];
    const double tau = tau_.get();
    double ap = 1.0, az = 1.0;
    const int64_t tot = D.n + D.p;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < D.n) {
            const double l = D.wl[i], u = D.wu[i], x = w[i];
            if (l > -INFINITY) {
                if (dw[i] < 0) ap = fmin(ap, -tau * (x - l) / dw[i]);
                if (dzl[i] < 0) az = fmin(az, -tau * zl[i] / dzl[i]);
            }
            if (u < INFINITY) {
                if (-dw[i] < 0) ap = fmin(ap, -tau * (u - x) / (-dw[i]));
                if (dzu[i] < 0) az = fmin(az, -tau * zu[i] / dzu[i]);
            }
        } else {
            const int64_t q = i - D.n;
            if (ds[q] < 0) ap = fmin(ap, -tau * s[q] / ds[q]);
            if (dzs[q] < 0) az = fmin(az, -tau * zs[q] / dzs[q]);
        }
    }
    double v;
    v = block_reduce(ap, 1, sh); if (threadIdx.x == 0) part[2 * blockIdx.x] = v;
    v = block_reduce(az, 1, sh); if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = v;
}

// ---- elementwise ---------------------------------------------------------
// split the KKT solution (natural order) into dw, dlam, dyc
__global__ void k_split(int64_t n_kkt, const int8_t *kind, const int64_t *index,
                        const double *sol, double *dw, double *dlam, double *dyc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_kkt) return;
    const int8_t k = kind[i];
    const int64_t j = index[i];
    if (k == 0) dw[j] = sol[i];
    else if (k == 1) dlam[j] = sol[i];
    else dyc[j] = sol[i];
}

// eliminated directions (recovery after eq. newtonsystem)
__global__ void k_recover(Dev D, const double *w, const double *r, const double *t,
                          const double *s, const double *lam, const double *yc, const double *zl,
                          const double *zu, const double *zs, const double *lam_n,
                          const double *nu0_n, DScalar rho_, DScalar mu_, const double *dw,
                          const double *dlam, const double *dyc, double *dr, double *dt,
                          double *ds, double *dzl, double *dzu, double *dzs) {
    const int64_t tot = D.n + D.m + D.p;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tot) return;
    const double rho = rho_.get(), mu = mu_.get();
    if (i < D.n) {
        const double l = D.wl[i], u = D.wu[i], x = w[i];
        dzl[i] = 0.0;
        dzu[i] = 0.0;
        if (l > -INFINITY) {
            const double sl = x - l;
            dzl[i] = mu / sl - zl[i] - zl[i] / sl * dw[i];
        }
        if (u < INFINITY) {
            const double su = u - x;
            dzu[i] = mu / su - zu[i] + zu[i] / su * dw[i];
        }
    } else if (i < D.n + D.m) {
        const int64_t j = i - D.n;
        dr[j] = (dlam[j] - (lam_n[j] + rho * r[j] - lam[j])) / rho;
    } else {
        const int64_t q = i - D.n - D.m;
        dt[q] = (dyc[q] - (nu0_n[q] + rho * t[q] - yc[q])) / rho;
        const double dsv = (mu / s[q] - yc[q] - dyc[q]) * s[q] / zs[q];
        ds[q] = dsv;
        dzs[q] = mu / s[q] - zs[q] - zs[q] / s[q] * dsv;
    }
}

// The trial point of every iterate vector in one launch: y = x + a d over
// the segments w, r, lam, t, s, yc (primal step a) and zs, zl, zu (dual step
// az).  With alpha != nullptr the two steps are read from the device (the
// fraction-to-boundary result), otherwise a and az are used.
struct StepSegs {
    const double *x[9];
    const double *d[9];
    double *y[9];
    int64_t end[9];   // cumulative lengths
    int dual_from;    // segments >= dual_from take az
};
__global__ void k_step_all(StepSegs S, double a, double az, const double *alpha) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.end[8]) return;
    int k = 0;
    while (i >= S.end[k]) k++;
    const int64_t j = i - (k ? S.end[k - 1] : 0);
    const double st = alpha ? alpha[k >= S.dual_from ? 1 : 0] : (k >= S.dual_from ? az : a);
    S.y[k][j] = S.x[k][j] + st * S.d[k][j];
}

// Fraction-to-boundary step lengths from the per-CTA partial minima
__global__ void k_ftb_finish(const double *part, int nblk, double *alpha) {
    __shared__ double sa[kT], sz[kT];
    double ap = 1.0, az = 1.0;
    for (int b = threadIdx.x; b < nblk; b += kT) {
        ap = fmin(ap, part[2 * b]);
        az = fmin(az, part[2 * b + 1]);
    }
    sa[threadIdx.x] = ap;
    sz[threadIdx.x] = az;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sa[threadIdx.x] = fmin(sa[threadIdx.x], sa[threadIdx.x + o]);
            sz[threadIdx.x] = fmin(sz[threadIdx.x], sz[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        alpha[0] = sa[0];
        alpha[1] = sz[0];
    }
}

// kappa_sigma safeguard of the bound multipliers (W&B 2006, eq. 16)
__global__ void k_zsafe(Dev D, const double *w, const double *s, double *zl, double *zu,
                        double *zs, DScalar mu_, double ks) {
    const int64_t tot = D.n + D.p;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tot) return;
    const double mu = mu_.get();
    if (i < D.n) {
        const double l = D.wl[i], u = D.wu[i], x = w[i];
        if (l > -INFINITY) {
            const double sl = x - l;
            zl[i] = fmax(fmin(zl[i], ks * mu / sl), mu / (ks * sl));
        }
        if (u < INFINITY) {
            const double su = u - x;
            zu[i] = fmax(fmin(zu[i], ks * mu / su), mu / (ks * su));
        }
    } else {
        const int64_t q = i - D.n;
        zs[q] = fmax(fmin(zs[q], ks * mu / s[q]), mu / (ks * s[q]));
    }
}

// t = w1 w2 + s
__global__ void k_reset_t(Dev D, const double *w, const double *s, double *t) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < D.p) t[q] = w[D.c1[q]] * w[D.c2[q]] + s[q];
}

inline int nb(int64_t n) { return (int)((n + kT - 1) / kT > 0 ? (n + kT - 1) / kT : 1); }

// ---- fixed-order combination of per-CTA partials ------------------------
// The host loop and the device-resident iteration combine the reductions'
// partials in the same order, so both take the same decisions from the same
// values: lane l of 32 folds entries l, l + 32, l + 64, ... in turn, then the
// 32 lane values are folded pairwise (l with l + 16 for l < 16, then l with
// l + 8, ..., l with l + 1).  Only additions, minima and maxima: no
// contraction into FMA can change a result.
enum { kOpMax = 0, kOpMin = 1, kOpSum = 2 };
__host__ __device__ inline double comb_ident(int op) {
    return op == kOpMax ? -INFINITY : (op == kOpMin ? INFINITY : 0.0);
}
__host__ __device__ inline double comb_op(double a, double b, int op) {
    return op == kOpMax ? fmax(a, b) : (op == kOpMin ? fmin(a, b) : a + b);
}
// entries p[b * stride], b < count
double comb32_host(const double *p, int count, int stride, int op) {
    double v[32];
    for (int l = 0; l < 32; l++) {
        double a = comb_ident(op);
        for (int b = l; b < count; b += 32) a = comb_op(a, p[(size_t)b * stride], op);
        v[l] = a;
    }
    for (int off = 16; off > 0; off >>= 1)
        for (int l = 0; l < off; l++) v[l] = comb_op(v[l], v[l + off], op);
    return v[0];
}
// the same in one warp (all 32 lanes call it; every lane gets the result)
__device__ double comb32_warp(const double *p, int count, int stride, int op) {
    const int l = threadIdx.x & 31;
    double a = comb_ident(op);
    for (int b = l; b < count; b += 32) a = comb_op(a, p[(size_t)b * stride], op);
    for (int off = 16; off > 0; off >>= 1) a = comb_op(a, __shfl_down_sync(0xffffffffu, a, off), op);
    return __shfl_sync(0xffffffffu, a, 0);
}

// Generation cost phi(w) = sum_g [c2 (100 p_g)^2 + c1 (100 p_g) + c0] / 1e4
// of eq. (scopf), per-generator terms folded in the order above.  Each term
// is ((c2 pv) pv + c1 pv) + c0 with pv = 100 p_g, rounded operation by
// operation on both sides.
struct GenCost {
    const double *c2, *c1, *c0;
    int ng;
};
double phi_fixed_host(const double *p0, const double *c2, const double *c1, const double *c0,
                      int ng) {
    std::vector<double> t(ng > 0 ? ng : 1);
    for (int i = 0; i < ng; i++) {
        const double pv = 100.0 * p0[i];
        t[i] = c2[i] * pv * pv + c1[i] * pv + c0[i];
    }
    return comb32_host(t.data(), ng, 1, kOpSum) / 1.0e4;
}
__device__ double phi_fixed_warp(const double *p0, const GenCost g) {
    const int l = threadIdx.x & 31;
    double a = 0.0;
    for (int i = l; i < g.ng; i += 32) {
        const double pv = __dmul_rn(100.0, p0[i]);
        const double t = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(g.c2[i], pv), pv),
                                             __dmul_rn(g.c1[i], pv)),
                                   g.c0[i]);
        a = a + t;
    }
    for (int off = 16; off > 0; off >>= 1) a = a + __shfl_down_sync(0xffffffffu, a, off);
    return __ddiv_rn(__shfl_sync(0xffffffffu, a, 0), 1.0e4);
}
// barrier function phi + (lam_n'r + rho/2 r'r) + (nu0_n't + rho/2 t't)
// - mu (sum ln slacks) from the 5-slot partials of k_barrier at `part`
__device__ double barrier_fixed_warp(double phi, double mu, const double *part) {
    const double bad = comb32_warp(part + 4, kB, 5, kOpSum);
    const double l0 = comb32_warp(part + 0, kB, 5, kOpSum), l1 = comb32_warp(part + 1, kB, 5, kOpSum);
    const double q2 = comb32_warp(part + 2, kB, 5, kOpSum), q3 = comb32_warp(part + 3, kB, 5, kOpSum);
    if (bad > 0) return INFINITY;
    return __dsub_rn(__dadd_rn(__dadd_rn(phi, q2), q3), __dmul_rn(mu, __dadd_rn(l0, l1)));
}

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double s() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

}  // namespace

constexpr int kPartSlots = 24;   // partial-sum slots per reduction block
int ipm_partials() { return kB * kPartSlots; }

// Whether the factorization of the assembled K at delta_w = 0 must report a
// zero pivot: one of the rows that receive no update in the elimination has
// a diagonal entry of exactly zero (its pivot is that entry, whatever the
// other values).  Only for a K assembled at delta_w = 0.
static bool zero_pivot_certain(scopf_handle *h) {
    if (h->n_lead == 0 || h->assembled_delta_w != 0.0) return false;
    if (h->lead_zero_valid) return h->lead_zero_host > 0;   // read with the norms
    launch_count_zero_diag(h->n_lead, h->lead_pdiag, h->pdiag_base, h->lead_zero, h->stream);
    int count = 0;
    cudaMemcpyAsync(&count, h->lead_zero, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    host_sync(h, h->stream);
    return count > 0;
}

// Inertia correction (W&B 2006, Alg. IC) around the factorization of the
// assembled K: IC-1 tries delta_w = 0 at every iteration, then delta_w grows
// from the IC-3 value until the inertia is (n, m + p, 0).  When the trial at
// 0 must meet a zero pivot (zero_pivot_certain) its outcome is known without
// factoring, and the correction starts at IC-3, as it would after factoring.
// K's primal diagonal is left shifted by the delta_w returned.
int factor_inertia(scopf_handle *h, int precision, double dw_last, double &delta, int &tries) {
    const scopf_options &o = h->opt;
    const int64_t npos = h->M.n, nneg = h->M.m + h->M.p;
    const double ic3 =
        dw_last == 0.0 ? o.delta_w0 : std::fmax(o.delta_w_min, o.kappa_w_minus * dw_last);
    delta = 0.0;
    if (o.known_zero_pivot && zero_pivot_certain(h)) {
        delta = ic3;
        h->n_known_zero++;
    }
    tries = 0;
    double current = h->assembled_delta_w;   // the shift of the assembled K
    while (true) {
        if (delta != current) {
            int r = set_delta_w(h, delta);
            if (r != SCOPF_OK) return r;
            current = delta;
        }
        int in[3];
        int r = factor_impl(h, precision, in);
        if (r != SCOPF_OK) return r;
        tries++;
        if (o.verbose >= 2)
            std::printf("    factor (%s) delta_w %.2e inertia (%d, %d, %d), want (%lld, %lld, 0)\n",
                        precision == SCOPF_PREC_MIXED ? "fp32" : "fp64", delta, in[0], in[1],
                        in[2], (long long)npos, (long long)nneg);
        if (in[0] == npos && in[1] == nneg && in[2] == 0) return SCOPF_OK;
        if (delta == 0.0)
            delta = ic3;
        else
            delta *= dw_last > 0.0 ? o.kappa_w_plus : o.kappa_w_plus_bar;
        if (delta > o.delta_w_max) return SCOPF_ERR_WRONG_INERTIA;
    }
}

// ===========================================================================
struct Ipm {
    scopf_handle *h;
    Dev D;
    const scopf_options &o;
    cudaStream_t s;
    std::vector<double> part;
    double *dpart = nullptr;
    int64_t n, m, p, n_il = 0, n_iu = 0;
    double *lam_trial_unused = nullptr;
    bool force_fp64 = false;
    int fallbacks = 0;

    // bound counts and the partial-sum buffer are set up once per handle
    explicit Ipm(scopf_handle *hh) : h(hh), o(hh->opt), s(hh->stream) {
        const Model &M = h->M;
        n = M.n;
        m = M.m;
        p = M.p;
        D = Dev{h->wl, h->wu, h->dm.comp1, h->dm.comp2, n, m, p};
        n_il = h->n_lower;
        n_iu = h->n_upper;
        part.resize(kB * kPartSlots);
        dpart = h->ipm_part;
    }

    // Several reductions write kB x k partials into consecutive regions of
    // dpart; one copy and one synchronisation bring them all to the host,
    // where each is combined in block order.
    void fetch(int k) {
        cudaMemcpyAsync(part.data(), dpart, sizeof(double) * kB * k, cudaMemcpyDeviceToHost, s);
        host_sync(h, s);
    }
    double comb(int k, int slot, int op, int region = 0) {
        return comb32_host(part.data() + (size_t)kB * region + slot, kB, k, op);
    }

    // ---- residual norms (error measure E_mu, W&B 2006 eq. 5)
    struct Norms {
        double dual, prim, cmin, cmax, ysum, zsum, theta, rmax, tmax;
        bool has_comp;
    };
    Norms norms(const scopf_state &st, double rho) {
        // regions: w (7 slots) at 0, constraint rows (5) at 7, pairs (9) at 12
        note_launch(), k_red_w<<<kB, kT, 0, s>>>(D, st.w, h->gw, st.zl, st.zu, dpart);
        note_launch(), k_red_m<<<kB, kT, 0, s>>>(D, h->c, st.r, st.lam, h->lam_n, rho, dpart + kB * 7);
        if (p)
            note_launch(), k_red_p<<<kB, kT, 0, s>>>(D, st.w, st.t, st.s, st.yc, st.zs, h->nu0_n, rho,
                                                      dpart + kB * 12);
        // the zero-pivot test of reading IC-1 (zero_pivot_certain) for the K
        // just assembled at delta_w = 0, in the same read-back
        const int regions = p ? 21 : 12;
        const bool zc = h->n_lead > 0 && h->assembled && h->assembled_delta_w == 0.0 &&
                        o.known_zero_pivot;
        int *zslot = reinterpret_cast<int *>(dpart + (size_t)kB * regions);
        if (zc) launch_count_zero_diag(h->n_lead, h->lead_pdiag, h->pdiag_base, zslot, s);
        fetch(regions + (zc ? 1 : 0));
        if (zc) {
            h->lead_zero_host = *reinterpret_cast<const int *>(part.data() + (size_t)kB * regions);
            h->lead_zero_valid = true;
        }
        return combine_norms();
    }
    // the norms from fetched partials: w (7 slots) at region 0, constraint
    // rows (5) at 7, pairs (9) at 12
    Norms combine_norms() {
        Norms N{};
        double dw = comb(7, 0, 0);
        double cmin = std::fmin(comb(7, 1, 1), comb(7, 3, 1));
        double cmax = std::fmax(comb(7, 2, 0), comb(7, 4, 0));
        double zsum = comb(7, 5, 2) + comb(7, 6, 2);
        double gr = comb(5, 0, 0, 7), pc = comb(5, 1, 0, 7), pcs = comb(5, 2, 2, 7),
               lsum = comb(5, 3, 2, 7);
        N.rmax = comb(5, 4, 0, 7);
        double gt = 0, gs = 0, py = 0, pys = 0, ycs = 0, zss = 0;
        N.tmax = 0;
        if (p) {
            gt = comb(9, 0, 0, 12);
            gs = comb(9, 1, 0, 12);
            py = comb(9, 2, 0, 12);
            pys = comb(9, 3, 2, 12);
            cmin = std::fmin(cmin, comb(9, 4, 1, 12));
            cmax = std::fmax(cmax, comb(9, 5, 0, 12));
            ycs = comb(9, 6, 2, 12);
            zss = comb(9, 7, 2, 12);
            N.tmax = comb(9, 8, 0, 12);
        }
        N.dual = std::fmax(std::fmax(dw, gr), std::fmax(gt, gs));
        N.prim = std::fmax(pc, py);
        N.cmin = cmin;
        N.cmax = cmax;
        N.has_comp = (n_il + n_iu + p) > 0;
        N.ysum = lsum + ycs;
        N.zsum = zsum + zss;
        N.theta = pcs + pys;
        return N;
    }
    double error(const Norms &N, double mu) const {
        const double nz = (double)(n_il + n_iu + p);
        const double sd = std::fmax(o.s_max, (N.ysum + N.zsum) / std::fmax(1.0, (double)(m + p) + nz)) / o.s_max;
        const double sc = std::fmax(o.s_max, N.zsum / std::fmax(1.0, nz)) / o.s_max;
        const double comp = N.has_comp ? std::fmax(N.cmax - mu, mu - N.cmin) : 0.0;
        return std::fmax(std::fmax(N.dual / sd, N.prim), comp / sc);
    }

    // objective phi(w) on the host from p_g^0
    double objective(const double *w) {
        double f = 0;
        scopf_eval(h, w, &f, nullptr, nullptr);
        return f;
    }
    // partials of k regions and p_g^0 of w in one copy + synchronisation
    std::vector<double> p0h;
    void fetch_p0(int k, const double *w) {
        const Model &M = h->M;
        p0h.resize(M.ng);
        cudaMemcpyAsync(part.data(), dpart, sizeof(double) * kB * k, cudaMemcpyDeviceToHost, s);
        if (M.ng)
            cudaMemcpyAsync(p0h.data(), w + M.border0, sizeof(double) * M.ng,
                            cudaMemcpyDeviceToHost, s);
        host_sync(h, s);
    }
    // phi from the fetched p_g^0 (the formula of scopf_eval, terms summed
    // in the fixed order)
    double phi_host() const {
        const Model &M = h->M;
        return phi_fixed_host(p0h.data(), M.c2.data(), M.c1.data(), M.c0.data(), M.ng);
    }
    // barrier function from its partials (5 slots at `region`)
    double barrier_value(double phi, double mu, int region) {
        if (comb(5, 4, 2, region) > 0) return INFINITY;
        return phi + comb(5, 2, 2, region) + comb(5, 3, 2, region) -
               mu * (comb(5, 0, 2, region) + comb(5, 1, 2, region));
    }
    // theta and the barrier function at a trial point, one round trip:
    // constraint rows at region 0 (5), pairs at 5 (9), barrier at 14 (5)
    void trial_eval(const scopf_state &st, double rho, double mu, double &theta, double &phib) {
        launch_eval_elements(h->dm, st.w, st.lam, st.yc, h->ev, 0, s);
        launch_constraints(h->dm, st.w, h->ev, h->c, s);
        note_launch(), k_red_m<<<kB, kT, 0, s>>>(D, h->c, st.r, st.lam, h->lam_n, 1.0, dpart);
        if (p)
            note_launch(), k_red_p<<<kB, kT, 0, s>>>(D, st.w, st.t, st.s, st.yc, st.zs, h->nu0_n, 1.0,
                                                      dpart + kB * 5);
        note_launch(), k_barrier<<<kB, kT, 0, s>>>(D, st.w, st.r, st.t, st.s, h->lam_n, h->nu0_n, rho,
                                                    dpart + kB * 14);
        fetch_p0(19, st.w);
        theta = comb(5, 2, 2) + (p ? comb(9, 3, 2, 5) : 0.0);
        phib = barrier_value(phi_host(), mu, 14);
    }
    void copy(scopf_state &dst, const scopf_state &src) {
        const int64_t len[9] = {n, m, p, p, m, p, n, n, p};
        double *const *a[9] = {&dst.w, &dst.r, &dst.t, &dst.s, &dst.lam, &dst.yc, &dst.zl, &dst.zu, &dst.zs};
        double *const *b[9] = {&src.w, &src.r, &src.t, &src.s, &src.lam, &src.yc, &src.zl, &src.zu, &src.zs};
        for (int i = 0; i < 9; i++)
            if (len[i]) cudaMemcpyAsync(*a[i], *b[i], sizeof(double) * len[i], cudaMemcpyDeviceToDevice, s);
    }

    // out = st + (a, az) d; alpha (device, 2 values) replaces (a, az) when given
    void step(scopf_state &out, const scopf_state &st, const scopf_state &d, double a, double az,
              const double *alpha = nullptr) {
        StepSegs S;
        const double *xs[9] = {st.w, st.r, st.lam, st.t, st.s, st.yc, st.zs, st.zl, st.zu};
        const double *ds[9] = {d.w, d.r, d.lam, d.t, d.s, d.yc, d.zs, d.zl, d.zu};
        double *ys[9] = {out.w, out.r, out.lam, out.t, out.s, out.yc, out.zs, out.zl, out.zu};
        const int64_t len[9] = {n, m, m, p, p, p, p, n, n};
        int64_t acc = 0;
        for (int k = 0; k < 9; k++) {
            S.x[k] = xs[k];
            S.d[k] = ds[k];
            S.y[k] = ys[k];
            acc += len[k];
            S.end[k] = acc;
        }
        S.dual_from = 6;
        if (acc > 0) note_launch(), k_step_all<<<nb(acc), kT, 0, s>>>(S, a, az, alpha);
    }

    // Newton direction with inertia correction; returns status, fills h->dir
    int direction(double &dw_last, double &delta, int &tries) {
        const int prec = force_fp64 ? SCOPF_PREC_FP64 : h->precision;
        int r = factor_inertia(h, prec, dw_last, delta, tries);
        if (r != SCOPF_OK) return r;
        double rel = 0;
        int steps = 0;
        r = solve_impl(h, h->rhs, h->sol, o.max_refine, &rel, &steps);
        if (r == SCOPF_ERR_REFINE_STALL && h->factored_precision == SCOPF_PREC_MIXED) {
            // FP32 factors no longer accurate enough: redo this step in FP64 and stay there
            force_fp64 = true;
            fallbacks++;
            int in[3];
            r = factor_impl(h, SCOPF_PREC_FP64, in);
            if (r != SCOPF_OK) return r;
            r = solve_impl(h, h->rhs, h->sol, o.max_refine, &rel, &steps);
        }
        if (r == SCOPF_ERR_REFINE_STALL) r = SCOPF_OK;  // FP64 factors: accept the refined step
        if (r != SCOPF_OK) return r;
        // cost switch: FP32 factors whose steps keep needing many refinement
        // steps cost more than FP64 factors (a factorization at the FP64 rate
        // against that many extra solves); switch after o.fp64_switch_streak
        // such steps in a row
        if (!force_fp64 && o.fp64_switch_refine > 0 && h->factored_precision == SCOPF_PREC_MIXED) {
            streak = steps >= o.fp64_switch_refine ? streak + 1 : 0;
            if (streak >= std::max(1, o.fp64_switch_streak)) {
                force_fp64 = true;
                fallbacks++;
            }
        }
        return SCOPF_OK;
    }
    int streak = 0;
};

// ===========================================================================
// Device-resident interior-point iteration (option ipm_graph).
//
// After the host has read the iteration's error measure and taken the
// barrier update, one iteration is two CUDA-graph launches:
//  * the direction graph (one per factor precision): right-hand side, then a
//    WHILE node over the inertia-correction trials (shift of the primal
//    diagonal, factorization, inertia test and next delta_w, W&B 2006 Alg. IC),
//    then -- an IF node on its success -- the solve and the refinement: a
//    WHILE node over FGMRES cycles whose Krylov steps are a nested WHILE node;
//  * the step graph: an IF node on a usable direction holding the recovery
//    of the eliminated directions, the fraction to the boundary, a WHILE node
//    over the filter line-search trials (trial point, its theta and barrier
//    function, the filter test and backtracking), an IF node for the elastic
//    restoration, the bound-multiplier safeguard, and the model evaluation,
//    KKT assembly and norm reductions at the new iterate.
// The host reads the norms' partials and the control block once per
// iteration.  The decisions are the host loop's, computed in the same
// order from the same partials (the fixed-order combination above), so the
// two loops take the same steps; the one difference is that the switching
// condition's (-grad'd)^s_phi is evaluated with CUDA's pow (the host loop
// uses the C library's; both within a few ulp).  A stalled FP32 refinement
// is handed to the host, which redoes the direction in FP64 (as the host
// loop does) and then launches the step graph.
namespace {

constexpr int kMaxIcTries = 200;   // safety bound only: delta_w > delta_w_max ends the loop first

template <typename T>
int dev_alloc(scopf_handle *h, size_t n, T **out) {
    T *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SCOPF_ERR_OOM : SCOPF_ERR_CUDA;
    }
    cudaMemset(p, 0, sizeof(T) * (n ? n : 1));
    h->allocations.push_back(p);
    *out = p;
    return SCOPF_OK;
}

__global__ void k_ctl_set(IpmCtl *c, double mu, double rho, double tau, double th, double tmin,
                          double tmax, double pow_th, double dw_last, int clear_filter) {
    c->mu = mu;
    c->rho = rho;
    c->tau = tau;
    c->th = th;
    c->theta_min = tmin;
    c->theta_max = tmax;
    c->pow_th = pow_th;
    c->dw_last = dw_last;
    if (clear_filter) c->filt_n = 0;
}

// the host redid the direction: the step graph may run
__global__ void k_ctl_ok(IpmCtl *c) {
    c->ok = 1;
    c->stall = 0;
    c->status = SCOPF_OK;
}

__global__ void k_cond_flag(cudaGraphConditionalHandle hc, const int *flag, int want) {
    cudaGraphSetConditional(hc, *flag == want ? 1u : 0u);
}

// IC-1 / IC-3 start: delta_w = 0, unless its factorization must meet an
// exactly zero pivot (counted into lead_zero), then the IC-3 value
__global__ void k_ic_start(IpmCtl *c, scopf_options o, int have_lead) {
    const double dw = c->dw_last;
    const double ic3 = dw == 0.0 ? o.delta_w0 : fmax(o.delta_w_min, __dmul_rn(o.kappa_w_minus, dw));
    c->ic3 = ic3;
    c->delta = 0.0;
    c->current = 0.0;   // the assembled K has delta_w = 0
    c->known_zero = 0;
    if (o.known_zero_pivot && have_lead && c->lead_zero > 0) {
        c->delta = ic3;
        c->known_zero = 1;
    }
    c->tries = 0;
    c->status = SCOPF_OK;
    c->ok = 0;
    c->stall = 0;
    c->dir_done = 0;
    c->ref_it = 0;
    c->ref_cycles = 0;
    c->rel = 0.0;
}

// K(delta_w): primal diagonal = (assembled entry) + delta_w
__global__ void k_diag_set_ctl(int64_t n, const int64_t *__restrict__ pos,
                               const double *__restrict__ base, const IpmCtl *__restrict__ c,
                               double *__restrict__ kval) {
    const double d = c->delta;
    if (d == c->current) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) kval[pos[i]] = base[i] + d;
}

// after a factorization: accept the inertia (n, m + p, 0) or take the next
// delta_w (IC-3 value, then growth by kappa_w_plus or kappa_w_plus_bar)
__global__ void k_ic_decide(IpmCtl *c, const FactorStatus *fs, scopf_options o, int64_t npos,
                            int64_t nneg, cudaGraphConditionalHandle loop) {
    c->current = c->delta;
    c->tries++;
    unsigned more = 0;
    if (fs->error) {
        c->status = SCOPF_ERR_TIMEOUT;
    } else if (!(fs->n_pos == npos && fs->n_neg == nneg && fs->n_zero == 0)) {
        const double d = c->delta == 0.0
                             ? c->ic3
                             : __dmul_rn(c->delta, c->dw_last > 0.0 ? o.kappa_w_plus : o.kappa_w_plus_bar);
        c->delta = d;
        if (d > o.delta_w_max || c->tries >= kMaxIcTries) c->status = SCOPF_ERR_WRONG_INERTIA;
        else more = 1;
    }
    cudaGraphSetConditional(loop, more);
}

// residual check of the refinement: red = (|b|_inf, |b - K x|_inf)
__global__ void k_ref_check(IpmCtl *c, const double *red, const KrylovCtl *kc, int first,
                            double tol, int max_refine, cudaGraphConditionalHandle loop) {
    const double bn = red[0], rn = red[1];
    if (first) {
        c->bden = bn > 0 ? bn : 1.0;
        c->ref_it = 0;
        c->ref_cycles = 0;
    } else {
        c->ref_it = kc->it;
        c->ref_cycles++;
    }
    c->bnorm = bn;
    const double r = rn / c->bden;
    c->rel = r;
    const bool more = r > tol && c->ref_it < max_refine && isfinite(r) &&
                      c->ref_cycles <= max_refine;
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// a new FGMRES cycle's Krylov loop (its WHILE node runs at least one step)
__global__ void k_kry_start_ctl(KrylovCtl *kc, const IpmCtl *c, int max_refine, double tol,
                                cudaGraphConditionalHandle kry) {
    kc->j = 0;
    kc->it = c->ref_it;
    kc->max_it = max_refine;
    kc->jend = 0;
    kc->target = __dmul_rn(__dmul_rn(tol, c->bnorm), 0.5);
    cudaGraphSetConditional(kry, 1u);
}

// outcome of the direction: a stalled FP32 refinement goes to the host,
// a stalled FP64 one is accepted
__global__ void k_ref_end(IpmCtl *c, const FactorStatus *fs, double tol, int mixed) {
    const double r = c->rel;
    c->dir_done = 1;
    if (fs->error) c->status = SCOPF_ERR_TIMEOUT;
    else if (!isfinite(r)) c->status = SCOPF_ERR_NUMERICAL;
    else if (r > tol && mixed) c->stall = 1;
    else c->ok = 1;
}

// Line search start (W&B 2006 Section 2.3): fraction-to-boundary steps from
// region 0 (2 slots), barrier function at the iterate from region 2 (5
// slots), its directional derivative from region 7 (5 slots), alpha_min
__global__ void k_ls_init(IpmCtl *c, const double *part, const double *p0, GenCost gc,
                          scopf_options o, cudaGraphConditionalHandle loop) {
    const double ap = fmin(1.0, comb32_warp(part, kB, 2, kOpMin));
    const double az = fmin(1.0, comb32_warp(part + 1, kB, 2, kOpMin));
    const double ph = barrier_fixed_warp(phi_fixed_warp(p0, gc), c->mu, part + kB * 2);
    const double gd = comb32_warp(part + kB * 7, kB * 5, 1, kOpSum);
    if (threadIdx.x != 0) return;
    const double th = c->th;
    double amin, pgd = 0.0;
    if (gd < 0) {
        pgd = pow(-gd, o.s_phi);
        amin = __dmul_rn(o.gamma_alpha,
                         fmin(o.gamma_theta, fmin(__ddiv_rn(__dmul_rn(o.gamma_phi, th), -gd),
                                                  __ddiv_rn(__dmul_rn(o.delta_sw, c->pow_th), pgd))));
    } else {
        amin = __dmul_rn(o.gamma_alpha, o.gamma_theta);
    }
    c->ph = ph;
    c->gd = gd;
    c->amin = amin;
    c->pow_gd = pgd;
    c->alpha[0] = ap;
    c->alpha[1] = az;
    c->nback = 0;
    c->accepted = 0;
    c->ftype = 0;
    c->trials = 0;
    cudaGraphSetConditional(loop, 1u);
}

// One line-search trial's verdict from the trial point's partials: theta
// from regions 0 (constraint rows, slot 2) and 5 (pairs, slot 3), barrier
// function from region 14.  Filter acceptance, switching condition,
// Armijo or sufficient decrease, backtracking by 1/2.
__global__ void k_ls_decide(IpmCtl *c, const double *part, const double *p0, GenCost gc,
                            double *filt, int filt_cap, scopf_options o, int has_p,
                            cudaGraphConditionalHandle loop) {
    const double tm = comb32_warp(part + 2, kB, 5, kOpSum);
    const double tp = has_p ? comb32_warp(part + kB * 5 + 3, kB, 9, kOpSum) : 0.0;
    const double tht = __dadd_rn(tm, tp);
    const double pht = barrier_fixed_warp(phi_fixed_warp(p0, gc), c->mu, part + kB * 14);
    const int lane = threadIdx.x & 31;
    const int nf = c->filt_n;
    bool in = false;
    for (int i = lane; i < nf; i += 32) in = in || (tht >= filt[2 * i] && pht >= filt[2 * i + 1]);
    in = __any_sync(0xffffffffu, in);
    if (lane != 0) return;
    const double a = c->alpha[0], th = c->th, ph = c->ph, gd = c->gd;
    bool ok = false, ftype = false;
    if (tht <= c->theta_max && !in) {
        const bool sw = gd < 0 && __dmul_rn(a, c->pow_gd) > __dmul_rn(o.delta_sw, c->pow_th);
        if (th <= c->theta_min && sw) {
            ok = pht <= __dadd_rn(ph, __dmul_rn(__dmul_rn(o.eta_phi, a), gd));
            ftype = ok;
        } else {
            ok = tht <= __dmul_rn(__dsub_rn(1.0, o.gamma_theta), th) ||
                 pht <= __dsub_rn(ph, __dmul_rn(o.gamma_phi, th));
        }
    }
    c->tht = tht;
    c->pht = pht;
    c->trials++;
    unsigned more = 0;
    if (ok) {
        c->accepted = 1;
        c->ftype = ftype;
        if (!ftype && nf < filt_cap) {
            filt[2 * nf] = __dmul_rn(__dsub_rn(1.0, o.gamma_theta), th);
            filt[2 * nf + 1] = __dsub_rn(ph, __dmul_rn(o.gamma_phi, th));
            c->filt_n = nf + 1;
        }
    } else {
        c->nback++;
        if (!(a < c->amin || c->nback >= o.max_backtrack) && c->trials <= o.max_backtrack + 1) {
            c->alpha[0] = __dmul_rn(a, 0.5);
            more = 1;
        }
    }
    cudaGraphSetConditional(loop, more);
}

__global__ void k_filter_clear(IpmCtl *c) { c->filt_n = 0; }

// st = trial, all nine iterate vectors
__global__ void k_copy_all(StepSegs S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.end[8]) return;
    int k = 0;
    while (i >= S.end[k]) k++;
    const int64_t j = i - (k ? S.end[k - 1] : 0);
    S.y[k][j] = S.x[k][j];
}

// ---- capture helpers
// a conditional handle on the graph stream `s` is capturing into (its
// default value is applied at every launch of the whole graph)
cudaError_t cond_handle(cudaStream_t s, unsigned dflt, cudaGraphConditionalHandle *hc) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    return cudaGraphConditionalHandleCreate(hc, g, dflt, cudaGraphCondAssignDefault);
}
// a conditional node after what `s` has captured so far; later work on `s`
// depends on it.  Its body graph is returned.
cudaError_t cond_node(cudaStream_t s, cudaGraphConditionalNodeType type,
                      cudaGraphConditionalHandle hc, cudaGraph_t *body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &ed, &nd);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, ed, nd, &np)) != cudaSuccess) return e;
    *body = np.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies);
}

// Streams of the capture, one per nesting level; h->stream follows the
// level being captured.
struct Capture {
    scopf_handle *h;
    cudaStream_t s[4] = {};
    cudaError_t e = cudaSuccess;
    cudaStream_t keep;
    bool timing;
    explicit Capture(scopf_handle *hh) : h(hh), keep(hh->stream), timing(hh->timer.on) {
        for (auto &x : s)
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        h->timer.on = false;
    }
    void chk(cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    }
    // start capturing level lv + 1 into `body`
    void open(int lv, cudaGraph_t body) {
        chk(cudaStreamBeginCaptureToGraph(s[lv + 1], body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed));
        h->stream = s[lv + 1];
    }
    void close(int lv) {
        cudaGraph_t g = nullptr;
        chk(cudaStreamEndCapture(s[lv + 1], &g));
        h->stream = s[lv];
    }
    ~Capture() {
        for (int lv = 3; lv >= 0; lv--) {   // end any capture an error left open
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (s[lv] && cudaStreamIsCapturing(s[lv], &cs) == cudaSuccess &&
                cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(s[lv], &g);
                if (lv == 0 && g) cudaGraphDestroy(g);
            }
        }
        for (auto &x : s)
            if (x) cudaStreamDestroy(x);
        cudaGetLastError();
        h->stream = keep;
        h->timer.on = timing;
    }
};

GenCost gen_cost(scopf_handle *h) {
    return GenCost{h->dm.c2, h->dm.c1, h->gen_c0, h->M.ng};
}

}  // namespace

void ipm_graphs_release(scopf_handle *h) {
    auto &G = h->ig;
    for (auto &x : G.dir)
        if (x) cudaGraphExecDestroy(x);
    if (G.step) cudaGraphExecDestroy(G.step);
    G.dir[0] = G.dir[1] = nullptr;
    G.step = nullptr;
}

namespace {

// The direction graph for factor precision T (see above).  cnt: kernels
// per launch of its parts -- [0] always, [1] per inertia trial, [2] once
// when the solve runs, [3] per refinement cycle, [4] per Krylov step.
template <typename T>
cudaError_t build_dir_graph(scopf_handle *h, cudaGraphExec_t *out, long long cnt[5]) {
    const scopf_options &o = h->opt;
    const Model &M = h->M;
    const int64_t n = M.n_kkt;
    constexpr int m = 16;
    const GmresLayout GL = gmres_layout(m);
    double *sc = h->kst + GL.sc;
    IpmCtl *c = h->ipm_ctl;
    const scopf_state &st = h->st;
    auto now = []() { return g_kernel_launches.load(); };
    const long long t0 = now();
    for (int i = 0; i < 5; i++) cnt[i] = 0;
    cudaGraph_t g = nullptr;
    const bool sinv_stale = h->sinv_stale;   // capturing the factorization sets it
    {
        Capture C(h);
        if (C.e != cudaSuccess) return C.e;
        C.chk(cudaStreamBeginCapture(C.s[0], cudaStreamCaptureModeRelaxed));
        h->stream = C.s[0];
        cudaStream_t s0 = C.s[0];
        {
            RhsArgs a{st.w, st.r, st.t, st.s, st.lam, st.yc, st.zs, h->gw, h->c,
                      h->lam_n, h->nu0_n, DScalar::at(&c->rho), DScalar::at(&c->mu)};
            launch_rhs(h->dm, a, h->rhs, s0);
        }
        const bool lead = h->n_lead > 0 && o.known_zero_pivot;
        if (lead) launch_count_zero_diag(h->n_lead, h->lead_pdiag, h->pdiag_base, &c->lead_zero, s0);
        note_launch(), k_ic_start<<<1, 1, 0, s0>>>(c, o, lead ? 1 : 0);
        cudaGraphConditionalHandle hic = 0, hok = 0, href = 0, hkry = 0;
        cudaGraph_t body = nullptr;
        // inertia correction: WHILE (default 1: at least one factorization)
        C.chk(cond_handle(s0, 1, &hic));
        if (C.e == cudaSuccess) C.chk(cond_node(s0, cudaGraphCondTypeWhile, hic, &body));
        if (C.e == cudaSuccess) {
            C.open(0, body);
            const long long t1 = now();
            if (h->n_pdiag)
                note_launch(), k_diag_set_ctl<<<nb(h->n_pdiag), kT, 0, C.s[1]>>>(
                    h->n_pdiag, h->pdiag_pos, h->pdiag_base, c, h->kval);
            C.chk(factor_enqueue<T>(h));
            note_launch(), k_ic_decide<<<1, 1, 0, C.s[1]>>>(c, h->fstat, o, M.n, M.m + M.p, hic);
            cnt[1] = now() - t1;
            C.close(0);
        }
        // solve and refinement: IF the inertia correction succeeded
        C.chk(cond_handle(s0, 0, &hok));
        note_launch(), k_cond_flag<<<1, 1, 0, s0>>>(hok, &c->status, SCOPF_OK);
        if (C.e == cudaSuccess) C.chk(cond_node(s0, cudaGraphCondTypeIf, hok, &body));
        if (C.e == cudaSuccess) {
            C.open(0, body);
            cudaStream_t s1 = C.s[1];
            const long long t3 = now();
            if (sizeof(T) == 4) launch_dense_inverse(h->S, (int)M.nborder, h->Sinv, s1);
            C.chk(cudaMemcpyAsync(h->res, h->rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s1));
            solve_once<T>(h, h->res, h->sol);
            launch_residual(h->dm, h->kval, h->sol, h->res, h->tmp_kkt, s1);
            reduce_maxabs2(h->res, h->tmp_kkt, n, h->red_out, h->red_scratch, s1);
            C.chk(cond_handle(s1, 0, &href));
            note_launch(), k_ref_check<<<1, 1, 0, s1>>>(c, h->red_out, h->kctl, 1, o.refine_tol,
                                                        o.max_refine, href);
            // FGMRES cycles: WHILE the residual is above refine_tol
            if (C.e == cudaSuccess) C.chk(cond_node(s1, cudaGraphCondTypeWhile, href, &body));
            if (C.e == cudaSuccess) {
                C.open(1, body);
                cudaStream_t s2 = C.s[2];
                const long long t4 = now();
                launch_multi_dot(h->tmp_kkt, n, 1, h->tmp_kkt, h->kpart, s2);
                launch_dot_finish(h->kpart, 1, sc + 0, true, s2);
                launch_gmres_init(h->kst, m, s2);
                launch_scale_inv(n, sc + 0, h->tmp_kkt, h->kv, s2);
                C.chk(cond_handle(s2, 0, &hkry));
                note_launch(), k_kry_start_ctl<<<1, 1, 0, s2>>>(h->kctl, c, o.max_refine,
                                                                o.refine_tol, hkry);
                // Krylov steps of the cycle: WHILE (set to 1 by the start kernel)
                if (C.e == cudaSuccess) C.chk(cond_node(s2, cudaGraphCondTypeWhile, hkry, &body));
                if (C.e == cudaSuccess) {
                    C.open(2, body);
                    cnt[4] = enqueue_krylov_step<T>(h, hkry);
                    C.close(2);
                }
                launch_kry_solve(h->kst, m, h->kctl, s2);
                launch_kry_axpy(h->sol, h->kz, n, h->kctl, true, h->kst + GL.c1, s2);
                launch_residual(h->dm, h->kval, h->sol, h->res, h->tmp_kkt, s2);
                reduce_maxabs2(h->res, h->tmp_kkt, n, h->red_out, h->red_scratch, s2);
                note_launch(), k_ref_check<<<1, 1, 0, s2>>>(c, h->red_out, h->kctl, 0,
                                                            o.refine_tol, o.max_refine, href);
                cnt[3] = now() - t4 - cnt[4];
                C.close(1);
            }
            note_launch(), k_ref_end<<<1, 1, 0, s1>>>(c, h->fstat, o.refine_tol, sizeof(T) == 4 ? 1 : 0);
            cnt[2] = now() - t3 - cnt[3] - cnt[4];
            C.close(0);
        }
        cnt[0] = now() - t0 - cnt[1] - cnt[2] - cnt[3] - cnt[4];
        C.chk(cudaGetLastError());
        if (C.e == cudaSuccess) C.chk(cudaStreamEndCapture(s0, &g));
        if (C.e == cudaSuccess) C.chk(cudaGraphInstantiate(out, g, 0));
        if (g) cudaGraphDestroy(g);
        g_kernel_launches -= now() - t0;   // counted when they run
        h->sinv_stale = sinv_stale;
        if (C.e != cudaSuccess) return C.e;
    }
    return cudaSuccess;
}

// y = x + alpha d over the nine iterate vectors (alpha on the device)
StepSegs step_segs(const scopf_state &out, const scopf_state &st, const scopf_state &d,
                   const Model &M) {
    StepSegs S;
    const double *xs[9] = {st.w, st.r, st.lam, st.t, st.s, st.yc, st.zs, st.zl, st.zu};
    const double *ds[9] = {d.w, d.r, d.lam, d.t, d.s, d.yc, d.zs, d.zl, d.zu};
    double *ys[9] = {out.w, out.r, out.lam, out.t, out.s, out.yc, out.zs, out.zl, out.zu};
    const int64_t len[9] = {M.n, M.m, M.m, M.p, M.p, M.p, M.p, M.n, M.n};
    int64_t acc = 0;
    for (int k = 0; k < 9; k++) {
        S.x[k] = xs[k];
        S.d[k] = ds[k];
        S.y[k] = ys[k];
        acc += len[k];
        S.end[k] = acc;
    }
    S.dual_from = 6;
    return S;
}

// The step graph (see above).  cnt: [0] always, [1] once when the direction
// is usable, [2] per line-search trial, [3] for a restoration.
cudaError_t build_step_graph(scopf_handle *h, cudaGraphExec_t *out, long long cnt[4]) {
    const scopf_options &o = h->opt;
    const Model &M = h->M;
    const int64_t n = M.n, m = M.m, p = M.p;
    IpmCtl *c = h->ipm_ctl;
    const scopf_state &st = h->st, &d = h->dir, &tr = h->trial;
    const Dev D{h->wl, h->wu, h->dm.comp1, h->dm.comp2, n, m, p};
    double *dpart = h->ipm_part;
    const DScalar rho = DScalar::at(&c->rho), mu = DScalar::at(&c->mu);
    const GenCost gc = gen_cost(h);
    const int filt_cap = o.max_inner + 2;
    auto now = []() { return g_kernel_launches.load(); };
    const long long t0 = now();
    for (int i = 0; i < 4; i++) cnt[i] = 0;
    cudaGraph_t g = nullptr;
    Capture C(h);
    if (C.e != cudaSuccess) return C.e;
    C.chk(cudaStreamBeginCapture(C.s[0], cudaStreamCaptureModeRelaxed));
    h->stream = C.s[0];
    cudaStream_t s0 = C.s[0];
    cudaGraphConditionalHandle hok = 0, hls = 0, hre = 0;
    cudaGraph_t body = nullptr;
    C.chk(cond_handle(s0, 0, &hok));
    note_launch(), k_cond_flag<<<1, 1, 0, s0>>>(hok, &c->ok, 1);
    if (C.e == cudaSuccess) C.chk(cond_node(s0, cudaGraphCondTypeIf, hok, &body));
    if (C.e == cudaSuccess) {
        C.open(0, body);
        cudaStream_t s1 = C.s[1];
        const long long t1 = now();
        note_launch(), k_split<<<nb(M.n_kkt), kT, 0, s1>>>(M.n_kkt, h->dm.row_kind, h->dm.row_index,
                                                           h->sol, d.w, d.lam, d.yc);
        note_launch(), k_recover<<<nb(n + m + p), kT, 0, s1>>>(D, st.w, st.r, st.t, st.s, st.lam, st.yc,
                                                                st.zl, st.zu, st.zs, h->lam_n, h->nu0_n,
                                                                rho, mu, d.w, d.lam, d.yc, d.r, d.t,
                                                                d.s, d.zl, d.zu, d.zs);
        note_launch(), k_ftb<<<kB, kT, 0, s1>>>(D, st.w, st.s, st.zl, st.zu, st.zs, d.w, d.s, d.zl,
                                                d.zu, d.zs, DScalar::at(&c->tau), dpart);
        note_launch(), k_barrier<<<kB, kT, 0, s1>>>(D, st.w, st.r, st.t, st.s, h->lam_n, h->nu0_n,
                                                    rho, dpart + kB * 2);
        note_launch(), k_dirderiv<<<kB, kT, 0, s1>>>(D, st.w, h->g, st.r, st.t, st.s, h->lam_n,
                                                     h->nu0_n, rho, mu, d.w, d.r, d.t, d.s,
                                                     dpart + kB * 7);
        C.chk(cond_handle(s1, 0, &hls));
        note_launch(), k_ls_init<<<1, 32, 0, s1>>>(c, dpart, st.w + M.border0, gc, o, hls);
        // line-search trials: WHILE (set to 1 by the start kernel)
        if (C.e == cudaSuccess) C.chk(cond_node(s1, cudaGraphCondTypeWhile, hls, &body));
        if (C.e == cudaSuccess) {
            C.open(1, body);
            cudaStream_t s2 = C.s[2];
            const long long t2 = now();
            const StepSegs S = step_segs(tr, st, d, M);
            if (S.end[8] > 0) note_launch(), k_step_all<<<nb(S.end[8]), kT, 0, s2>>>(S, 0.0, 0.0, c->alpha);
            launch_eval_elements(h->dm, tr.w, tr.lam, tr.yc, h->ev, 0, s2);
            launch_constraints(h->dm, tr.w, h->ev, h->c, s2);
            note_launch(), k_red_m<<<kB, kT, 0, s2>>>(D, h->c, tr.r, tr.lam, h->lam_n, 1.0, dpart);
            if (p)
                note_launch(), k_red_p<<<kB, kT, 0, s2>>>(D, tr.w, tr.t, tr.s, tr.yc, tr.zs, h->nu0_n,
                                                          1.0, dpart + kB * 5);
            note_launch(), k_barrier<<<kB, kT, 0, s2>>>(D, tr.w, tr.r, tr.t, tr.s, h->lam_n, h->nu0_n,
                                                        rho, dpart + kB * 14);
            note_launch(), k_ls_decide<<<1, 32, 0, s2>>>(c, dpart, tr.w + M.border0, gc, h->ipm_filter,
                                                         filt_cap, o, p > 0 ? 1 : 0, hls);
            cnt[2] = now() - t2;
            C.close(1);
        }
        // restoration: IF no trial was accepted
        C.chk(cond_handle(s1, 0, &hre));
        note_launch(), k_cond_flag<<<1, 1, 0, s1>>>(hre, &c->accepted, 0);
        if (C.e == cudaSuccess) C.chk(cond_node(s1, cudaGraphCondTypeIf, hre, &body));
        if (C.e == cudaSuccess) {
            C.open(1, body);
            cudaStream_t s2 = C.s[2];
            const long long t2 = now();
            const StepSegs S = step_segs(tr, st, d, M);
            if (S.end[8] > 0) note_launch(), k_step_all<<<nb(S.end[8]), kT, 0, s2>>>(S, 0.0, 0.0, c->alpha);
            launch_eval_elements(h->dm, tr.w, tr.lam, tr.yc, h->ev, 0, s2);
            launch_constraints(h->dm, tr.w, h->ev, tr.r, s2);
            if (p) note_launch(), k_reset_t<<<nb(p), kT, 0, s2>>>(D, tr.w, tr.s, tr.t);
            note_launch(), k_filter_clear<<<1, 1, 0, s2>>>(c);
            cnt[3] = now() - t2;
            C.close(1);
        }
        note_launch(), k_zsafe<<<nb(n + p), kT, 0, s1>>>(D, tr.w, tr.s, tr.zl, tr.zu, tr.zs, mu,
                                                         o.kappa_sigma);
        {
            const StepSegs S = step_segs(st, tr, d, M);   // st = trial
            if (S.end[8] > 0) note_launch(), k_copy_all<<<nb(S.end[8]), kT, 0, s1>>>(S);
        }
        // the next iterate's model, KKT (delta_w = 0) and norm partials
        assemble_enqueue(h, &st, rho, 0.0);
        note_launch(), k_red_w<<<kB, kT, 0, s1>>>(D, st.w, h->gw, st.zl, st.zu, dpart);
        note_launch(), k_red_m<<<kB, kT, 0, s1>>>(D, h->c, st.r, st.lam, h->lam_n, rho, dpart + kB * 7);
        if (p)
            note_launch(), k_red_p<<<kB, kT, 0, s1>>>(D, st.w, st.t, st.s, st.yc, st.zs, h->nu0_n, rho,
                                                      dpart + kB * 12);
        cnt[1] = now() - t1 - cnt[2] - cnt[3];
        C.close(0);
    }
    cnt[0] = now() - t0 - cnt[1] - cnt[2] - cnt[3];
    C.chk(cudaGetLastError());
    if (C.e == cudaSuccess) C.chk(cudaStreamEndCapture(s0, &g));
    if (C.e == cudaSuccess) C.chk(cudaGraphInstantiate(out, g, 0));
    if (g) cudaGraphDestroy(g);
    g_kernel_launches -= now() - t0;
    return C.e;
}

}  // namespace

namespace {

// Allocations and graphs of the device-resident iteration for factor
// precision `prec`; G.failed (with last_error) when a graph could not be
// built -- the host loop then runs.
int ipm_graph_setup(scopf_handle *h, int prec) {
    auto &G = h->ig;
    if (G.failed) return SCOPF_OK;
    const Model &M = h->M;
    if (!h->ipm_ctl) {
        int r = dev_alloc(h, 1, &h->ipm_ctl);
        if (r == SCOPF_OK) r = dev_alloc(h, 2 * (size_t)(h->opt.max_inner + 2), &h->ipm_filter);
        if (r == SCOPF_OK) r = dev_alloc(h, (size_t)M.ng, &h->gen_c0);
        if (r != SCOPF_OK) return r;
        if (M.ng && cudaMemcpy(h->gen_c0, M.c0.data(), sizeof(double) * M.ng,
                               cudaMemcpyHostToDevice) != cudaSuccess)
            return SCOPF_ERR_CUDA;
    }
    int r = krylov_buffers(h);
    if (r != SCOPF_OK) return r;
    if (h->ig_stale || G.key_st != h->st.w || G.key_trial != h->trial.w) {
        ipm_graphs_release(h);   // built around other buffers
        h->ig_stale = false;
    }
    G.key_st = h->st.w;
    G.key_trial = h->trial.w;
    const int pi = prec == SCOPF_PREC_MIXED ? 0 : 1;
    cudaError_t e = cudaSuccess;
    if (!G.dir[pi]) {
        long long cnt[5];
        e = pi == 0 ? build_dir_graph<float>(h, &G.dir[pi], cnt)
                    : build_dir_graph<double>(h, &G.dir[pi], cnt);
        if (e == cudaSuccess) {
            G.k_dir_pre[pi] = cnt[0];
            G.k_ic[pi] = cnt[1];
            G.k_solve[pi] = cnt[2];
            G.k_ref[pi] = cnt[3];
            G.k_kry[pi] = cnt[4];
        } else {
            G.dir[pi] = nullptr;
        }
    }
    if (e == cudaSuccess && !G.step) {
        long long cnt[4];
        e = build_step_graph(h, &G.step, cnt);
        if (e == cudaSuccess) {
            G.k_step_pre = cnt[0];
            G.k_step_if = cnt[1];
            G.k_ls = cnt[2];
            G.k_restore = cnt[3];
        } else {
            G.step = nullptr;
        }
    }
    if (e != cudaSuccess) {
        h->last_error = std::string("interior-point iteration graph: ") + cudaGetErrorString(e);
        G.failed = true;
        ipm_graphs_release(h);
    }
    return SCOPF_OK;
}

// kernels the iteration's graph launches ran (the launch count)
long long graph_kernels(const scopf_handle *h, int pi, const IpmCtl &c, bool step_ran) {
    const auto &G = h->ig;
    long long k = G.k_dir_pre[pi] + G.k_ic[pi] * c.tries;
    if (c.dir_done) k += G.k_solve[pi] + G.k_ref[pi] * c.ref_cycles + G.k_kry[pi] * c.ref_it;
    k += G.k_step_pre;
    if (step_ran) k += G.k_step_if + G.k_ls * c.trials + (c.accepted ? 0 : G.k_restore);
    return k;
}

}  // namespace

// One device-resident iteration at (mu, rho): the direction and step graphs
// and one read-back of the control block (into `out`) and of the new
// iterate's norm partials (into I.part).  Returns the direction's error, if
// any.
static int graph_iteration(Ipm &I, int prec, double mu, double rho, double tau, double th,
                           double theta_min, double theta_max, double dw_last, bool clear_filter,
                           IpmCtl &out) {
    scopf_handle *h = I.h;
    const scopf_options &o = h->opt;
    cudaStream_t s = h->stream;
    auto &G = h->ig;
    const int pi = prec == SCOPF_PREC_MIXED ? 0 : 1;
    const int regions = I.p ? 21 : 12;
    note_launch(), k_ctl_set<<<1, 1, 0, s>>>(h->ipm_ctl, mu, rho, tau, th, theta_min, theta_max,
                                             std::pow(th, o.s_theta), dw_last, clear_filter ? 1 : 0);
    cudaError_t e = cudaGraphLaunch(G.dir[pi], s);
    if (e == cudaSuccess) e = cudaGraphLaunch(G.step, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(I.part.data(), I.dpart, sizeof(double) * kB * regions,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&out, h->ipm_ctl, sizeof(IpmCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = host_sync(h, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return SCOPF_ERR_CUDA;
    }
    g_kernel_launches += graph_kernels(h, pi, out, out.ok != 0);
    h->n_factor += out.tries;
    h->n_known_zero += out.known_zero;
    h->factored_precision = prec;
    h->last_delta_w = out.delta;
    if (out.dir_done) {
        h->n_refine += out.ref_it;
        h->n_solve_calls++;
    }
    if (out.status != SCOPF_OK) {
        if (out.status == SCOPF_ERR_TIMEOUT)
            h->last_error = "dependency wait timed out in the factorization or a sweep";
        return out.status;
    }
    if (out.stall) {
        // FP32 factors no longer accurate enough: redo the direction with
        // FP64 factors (host-driven, as in the host loop) and stay in FP64
        I.force_fp64 = true;
        I.fallbacks++;
        int in[3];
        int r = factor_impl(h, SCOPF_PREC_FP64, in);
        if (r != SCOPF_OK) return r;
        double rel = 0;
        int steps = 0;
        r = solve_impl(h, h->rhs, h->sol, o.max_refine, &rel, &steps);
        if (r == SCOPF_ERR_REFINE_STALL) r = SCOPF_OK;
        if (r != SCOPF_OK) return r;
        note_launch(), k_ctl_ok<<<1, 1, 0, s>>>(h->ipm_ctl);
        e = cudaGraphLaunch(G.step, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(I.part.data(), I.dpart, sizeof(double) * kB * regions,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&out, h->ipm_ctl, sizeof(IpmCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = host_sync(h, s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            h->last_error = cudaGetErrorString(e);
            return SCOPF_ERR_CUDA;
        }
        g_kernel_launches += h->ig.k_step_pre + h->ig.k_step_if + h->ig.k_ls * out.trials +
                             (out.accepted ? 0 : h->ig.k_restore);
    } else if (!I.force_fp64 && o.fp64_switch_refine > 0 && prec == SCOPF_PREC_MIXED) {
        // the cost switch of the host loop (Ipm::direction)
        I.streak = out.ref_it >= o.fp64_switch_refine ? I.streak + 1 : 0;
        if (I.streak >= std::max(1, o.fp64_switch_streak)) {
            I.force_fp64 = true;
            I.fallbacks++;
        }
    }
    // the direction graph formed S^-1 of its factors; the step graph
    // assembled K at the new iterate (delta_w = 0)
    h->sinv_stale = false;
    h->assembled = true;
    h->factored = false;
    h->lead_zero_valid = false;
    h->last_delta_w = 0.0;
    h->assembled_delta_w = 0.0;
    h->last_rho = rho;
    return SCOPF_OK;
}

int ncl_solve_impl(scopf_handle *h, const scopf_state *warm, scopf_result *res, bool resume) {
    Timer T;
    const scopf_options &o = h->opt;
    const Model &M = h->M;
    cudaStream_t s = h->stream;
    Ipm I(h);
    const int64_t n = M.n, m = M.m, p = M.p;
    Dev D = I.D;
    scopf_state &st = h->st;
    scopf_state &d = h->dir;
    scopf_state &tr = h->trial;
    double rho = resume ? h->rho : o.rho_init;
    if (!resume) {
        cudaMemsetAsync(h->lam_n, 0, sizeof(double) * (m ? m : 1), s);
        cudaMemsetAsync(h->nu0_n, 0, sizeof(double) * (p ? p : 1), s);
    }
    if (resume) {
        // continue from the handle's iterate and NCL parameters (a checkpoint)
    } else if (warm) {
        int r = scopf_load_state(h, warm);
        if (r != SCOPF_OK) return r;
    } else {
        // flat start, bound push (W&B 2006 Section 3.6), NCL multiplier identities
        std::vector<double> w = M.w_init;
        for (int64_t q = 0; q < p; q++) w[M.comp1[q]] = std::fmax(w[M.comp1[q]], o.comp_init);
        std::vector<double> wl(n), wu(n), zl(n, 0.0), zu(n, 0.0);
        cudaMemcpy(wl.data(), h->wl, sizeof(double) * n, cudaMemcpyDeviceToHost);
        cudaMemcpy(wu.data(), h->wu, sizeof(double) * n, cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < n; i++) {
            const bool hl = std::isfinite(wl[i]), hu = std::isfinite(wu[i]);
            double pl = hl ? o.bound_push * std::fmax(1.0, std::fabs(wl[i])) : 0.0;
            double pu = hu ? o.bound_push * std::fmax(1.0, std::fabs(wu[i])) : 0.0;
            if (hl && hu) {
                pl = std::fmin(pl, o.bound_frac * (wu[i] - wl[i]));
                pu = std::fmin(pu, o.bound_frac * (wu[i] - wl[i]));
            }
            if (hl) w[i] = std::fmax(w[i], wl[i] + pl);
            if (hu) w[i] = std::fmin(w[i], wu[i] - pu);
            if (hl) zl[i] = 1.0;
            if (hu) zu[i] = 1.0;
        }
        std::vector<double> sv(p, o.slack_init), t(p), yc(p);
        for (int64_t q = 0; q < p; q++) {
            t[q] = w[M.comp1[q]] * w[M.comp2[q]] + sv[q];
            yc[q] = o.rho_init * t[q];
        }
        cudaMemcpy(st.w, w.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
        cudaMemcpy(st.zl, zl.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
        cudaMemcpy(st.zu, zu.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
        if (p) {
            cudaMemcpy(st.s, sv.data(), sizeof(double) * p, cudaMemcpyHostToDevice);
            cudaMemcpy(st.t, t.data(), sizeof(double) * p, cudaMemcpyHostToDevice);
            cudaMemcpy(st.yc, yc.data(), sizeof(double) * p, cudaMemcpyHostToDevice);
            cudaMemcpy(st.zs, yc.data(), sizeof(double) * p, cudaMemcpyHostToDevice);
        }
        // r = c(w), lam = rho_init r
        launch_eval_elements(h->dm, st.w, st.lam, st.yc, h->ev, 0, s);
        launch_constraints(h->dm, st.w, h->ev, st.r, s);
        cudaMemsetAsync(st.lam, 0, sizeof(double) * (m ? m : 1), s);
        launch_axpy(m, o.rho_init, st.r, st.lam, s);
        host_sync(h, s);
    }
    double mu = o.mu_init, eta = o.eta_init, omega = o.omega_init, dw_last = 0.0;
    if (resume) {
        mu = h->mu_last;
        eta = h->eta_last;
        omega = h->omega_last;
        dw_last = h->dw_last;
    }
    int status = SCOPF_ERR_MAX_ITER;
    int outer = 0, inner = 0;
    bool inner_limit = false;
    h->hist_inner.clear();
    h->hist_outer.clear();
    double E0 = INFINITY, feas = INFINITY;
    double t_newton = 0.0;
    const int fact0 = h->n_factor, ref0 = h->n_refine;
    const long long syncs0 = h->n_host_syncs;
    int graph_iters = 0;
    for (outer = 1; outer <= o.max_outer; outer++) {
        const double om = std::fmax(omega, o.tol);
        // ------------------------------------------------------------ inner
        int r = assemble_impl(h, &st, h->lam_n, h->nu0_n, rho, mu, 0.0, nullptr);
        if (r != SCOPF_OK) return r;
        Ipm::Norms N = I.norms(st, rho);
        const double th0 = N.theta;
        const double theta_max = 1e4 * std::fmax(1.0, th0), theta_min = 1e-4 * std::fmax(1.0, th0);
        std::vector<std::pair<double, double>> filt;
        bool clear_filter = true;   // the device-resident iteration's filter starts empty
        int inner_status = SCOPF_OK;
        while (true) {
            E0 = I.error(N, o.fixed_mu ? mu : 0.0);   // fixed mu: the barrier error
            if (E0 <= om) break;
            if (inner >= o.max_inner) {
                inner_status = SCOPF_ERR_MAX_ITER;
                break;
            }
            double Emu = I.error(N, mu);
            while (!o.fixed_mu && Emu <= o.kappa_eps * mu && mu > o.mu_min) {
                mu = std::fmax(o.mu_min, std::fmin(o.kappa_mu * mu, std::pow(mu, o.theta_mu)));
                filt.clear();
                clear_filter = true;
                Emu = I.error(N, mu);
            }
            const double tau = std::fmax(o.tau_min, 1.0 - mu);
            const bool graph = o.ipm_graph && o.device_loop;
            if (graph) {
                const int prec = I.force_fp64 ? SCOPF_PREC_FP64 : h->precision;
                r = ipm_graph_setup(h, prec);
                if (r != SCOPF_OK) return r;
            }
            if (graph && !h->ig.failed) {
                // the iteration as two graph launches and one read-back
                Timer tn;
                const int prec = I.force_fp64 ? SCOPF_PREC_FP64 : h->precision;
                const int fact_before = h->n_factor, refine_before = h->n_refine;
                const double E0_step = E0, th = N.theta;
                IpmCtl c{};
                r = graph_iteration(I, prec, mu, rho, tau, th, theta_min, theta_max, dw_last,
                                    clear_filter, c);
                clear_filter = false;
                if (r != SCOPF_OK) {
                    inner_status = r == SCOPF_ERR_WRONG_INERTIA ? SCOPF_ERR_NUMERICAL : r;
                    break;
                }
                if (c.delta > 0.0) dw_last = c.delta;
                inner++;
                graph_iters++;
                N = I.combine_norms();
                const double it_s = tn.s();
                t_newton += it_s;
                const double rec[kHistInner] = {(double)outer, (double)inner, mu, rho, E0_step, th,
                                                c.ph, c.alpha[0], c.alpha[1], c.delta,
                                                (double)(h->n_factor - fact_before),
                                                (double)(h->n_refine - refine_before),
                                                (double)h->factored_precision,
                                                c.accepted ? 1.0 : 0.0, (double)c.nback,
                                                it_s * 1e3};
                h->hist_inner.insert(h->hist_inner.end(), rec, rec + kHistInner);
                if (o.verbose)
                    std::printf("  it %4d mu %.1e E0 %.2e th %.2e a %.2e dw %.1e tries %d%s (graph)\n",
                                inner, mu, E0, th, c.alpha[0], c.delta, c.tries,
                                c.accepted ? "" : " R");
                continue;
            }
            Timer tn;
            // right-hand side at the final mu (K at delta_w = 0 is assembled)
            {
                RhsArgs a{st.w, st.r, st.t, st.s, st.lam, st.yc, st.zs, h->gw, h->c,
                          h->lam_n, h->nu0_n, rho, mu};
                launch_rhs(h->dm, a, h->rhs, s);
            }
            double delta = 0.0;
            int tries = 0;
            const int fact_before = h->n_factor, refine_before = h->n_refine;
            const double E0_step = E0;
            r = I.direction(dw_last, delta, tries);
            if (r != SCOPF_OK) {
                inner_status = r == SCOPF_ERR_WRONG_INERTIA ? SCOPF_ERR_NUMERICAL : r;
                break;
            }
            if (delta > 0.0) dw_last = delta;
            // split + recover
            note_launch(), k_split<<<nb(M.n_kkt), kT, 0, s>>>(M.n_kkt, h->dm.row_kind, h->dm.row_index, h->sol,
                                               d.w, d.lam, d.yc);
            note_launch(), k_recover<<<nb(n + m + p), kT, 0, s>>>(D, st.w, st.r, st.t, st.s, st.lam, st.yc,
                                                   st.zl, st.zu, st.zs, h->lam_n, h->nu0_n, rho,
                                                   mu, d.w, d.lam, d.yc, d.r, d.t, d.s, d.zl,
                                                   d.zu, d.zs);
            // fraction to the boundary (region 0, 2 slots), barrier function at
            // the current point (region 2, 5 slots) and its directional
            // derivative (region 7, 5 slots; h->g holds grad phi): one round trip
            note_launch(), k_ftb<<<kB, kT, 0, s>>>(D, st.w, st.s, st.zl, st.zu, st.zs, d.w, d.s, d.zl, d.zu,
                                    d.zs, tau, I.dpart);
            note_launch(), k_barrier<<<kB, kT, 0, s>>>(D, st.w, st.r, st.t, st.s, h->lam_n, h->nu0_n, rho,
                                                        I.dpart + kB * 2);
            note_launch(), k_dirderiv<<<kB, kT, 0, s>>>(D, st.w, h->g, st.r, st.t, st.s, h->lam_n, h->nu0_n, rho,
                                         mu, d.w, d.r, d.t, d.s, I.dpart + kB * 7);
            I.fetch_p0(12, st.w);
            const double ap = std::fmin(1.0, I.comb(2, 0, kOpMin));
            const double az = std::fmin(1.0, I.comb(2, 1, kOpMin));
            const double th = N.theta;
            const double ph = I.barrier_value(I.phi_host(), mu, 2);
            const double gd = comb32_host(I.part.data() + (size_t)kB * 7, kB * 5, 1, kOpSum);
            double amin;
            if (gd < 0)
                amin = o.gamma_alpha * std::fmin(o.gamma_theta, std::fmin(o.gamma_phi * th / -gd,
                        o.delta_sw * std::pow(th, o.s_theta) / std::pow(-gd, o.s_phi)));
            else
                amin = o.gamma_alpha * o.gamma_theta;
            double a = ap;
            bool accepted = false, ftype = false;
            int nback = 0;
            while (true) {
                I.step(tr, st, d, a, az);
                double tht, pht;
                I.trial_eval(tr, rho, mu, tht, pht);
                bool ok = false;
                ftype = false;
                bool in_filter = false;
                for (auto &fp : filt)
                    if (tht >= fp.first && pht >= fp.second) {
                        in_filter = true;
                        break;
                    }
                if (tht <= theta_max && !in_filter) {
                    const bool sw = gd < 0 && a * std::pow(-gd, o.s_phi) > o.delta_sw * std::pow(th, o.s_theta);
                    if (th <= theta_min && sw) {
                        ok = pht <= ph + o.eta_phi * a * gd;
                        ftype = ok;
                    } else {
                        ok = tht <= (1 - o.gamma_theta) * th || pht <= ph - o.gamma_phi * th;
                    }
                }
                if (ok) {
                    accepted = true;
                    break;
                }
                nback++;
                if (a < amin || nback >= o.max_backtrack) break;
                a *= 0.5;
            }
            if (!accepted) {
                // elastic reset: r and t absorb the violation (NCL restoration)
                I.step(tr, st, d, a, az);
                launch_eval_elements(h->dm, tr.w, tr.lam, tr.yc, h->ev, 0, s);
                launch_constraints(h->dm, tr.w, h->ev, tr.r, s);
                if (p) note_launch(), k_reset_t<<<nb(p), kT, 0, s>>>(D, tr.w, tr.s, tr.t);
                filt.clear();
            } else if (!ftype) {
                filt.push_back({(1 - o.gamma_theta) * th, ph - o.gamma_phi * th});
            }
            note_launch(), k_zsafe<<<nb(n + p), kT, 0, s>>>(D, tr.w, tr.s, tr.zl, tr.zu, tr.zs, mu, o.kappa_sigma);
            std::swap(st, tr);
            inner++;
            if (o.verbose)
                std::printf("  it %4d mu %.1e E0 %.2e th %.2e a %.2e dw %.1e tries %d%s\n", inner, mu,
                            E0, th, a, delta, tries, accepted ? "" : " R");
            r = assemble_impl(h, &st, h->lam_n, h->nu0_n, rho, mu, 0.0, nullptr);
            if (r != SCOPF_OK) return r;
            N = I.norms(st, rho);   // waits for the step (and this assembly)
            const double it_s = tn.s();
            t_newton += it_s;
            {
                const double rec[kHistInner] = {(double)outer, (double)inner, mu, rho, E0_step, th, ph,
                                                a, az, delta, (double)(h->n_factor - fact_before),
                                                (double)(h->n_refine - refine_before),
                                                (double)h->factored_precision, accepted ? 1.0 : 0.0,
                                                (double)nback, it_s * 1e3};
                h->hist_inner.insert(h->hist_inner.end(), rec, rec + kHistInner);
            }
        }
        feas = std::fmax(N.rmax, N.tmax);
        {
            const double rec[kHistOuter] = {(double)outer, rho, N.rmax, N.tmax, E0, eta, omega,
                                            (double)inner};
            h->hist_outer.insert(h->hist_outer.end(), rec, rec + kHistOuter);
        }
        if (o.verbose)
            std::printf("outer %d rho %.1e |r,t| %.2e E0 %.2e inner %d\n", outer, rho, feas, E0, inner);
        if (inner_status != SCOPF_OK) {
            status = inner_status;
            inner_limit = inner_status == SCOPF_ERR_MAX_ITER;
            break;
        }
        if (feas <= std::fmax(eta, o.tol)) {
            if (feas <= o.tol && E0 <= o.tol) {
                status = SCOPF_OK;
                break;
            }
            launch_axpy(m, rho, st.r, h->lam_n, s);
            launch_axpy(p, rho, st.t, h->nu0_n, s);
            eta = std::fmax(eta / 10.0, o.tol);
            omega = std::fmax(omega / 10.0, o.tol);
        } else {
            if (rho * 10.0 > o.rho_max) {
                status = SCOPF_ERR_INFEASIBLE;
                break;
            }
            if (h->screen_blocks) {
                // batched screening: blocks within eta update their multipliers
                r = block_multiplier_update(h, rho, std::fmax(eta, o.tol));
                if (r != SCOPF_OK) return r;
            }
            rho *= 10.0;
        }
    }
    if (outer > o.max_outer) outer = o.max_outer;
    host_sync(h, s);
    h->rho = rho;
    h->mu_last = mu;
    h->dw_last = dw_last;
    h->eta_last = eta;
    h->omega_last = omega;
    h->have_ncl = true;
    h->has_solution = status == SCOPF_OK;
    h->inner_limit = inner_limit;
    // final report
    res->status = status;
    res->outer_iters = outer;
    res->inner_iters = inner;
    res->factorizations = h->n_factor - fact0;
    res->refine_steps = h->n_refine - ref0;
    res->fp64_fallbacks = I.fallbacks;
    res->objective = I.objective(st.w);
    res->kkt_error = E0;
    res->feas_rt = feas;
    // violation of eq. (mpcc): |c|, bound and complementarity violations
    {
        launch_eval_elements(h->dm, st.w, st.lam, st.yc, h->ev, 0, s);
        launch_constraints(h->dm, st.w, h->ev, h->c, s);
        double v = device_maxabs(h, h->c, m);
        std::vector<double> w(n), wl(M.wl), wu(M.wu);
        cudaMemcpy(w.data(), st.w, sizeof(double) * n, cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < n; i++) {
            if (std::isfinite(wl[i])) v = std::fmax(v, wl[i] - w[i]);
            if (std::isfinite(wu[i])) v = std::fmax(v, w[i] - wu[i]);
        }
        for (int64_t q = 0; q < p; q++) v = std::fmax(v, std::fabs(w[M.comp1[q]] * w[M.comp2[q]]));
        res->max_violation = v;
    }
    res->rho = rho;
    res->mu = mu;
    res->time_total_s = T.s();
    res->time_newton_s = t_newton;
    res->delta_w_last = dw_last;
    res->host_round_trips = h->n_host_syncs - syncs0;
    res->graph_iters = graph_iters;
    return status == SCOPF_OK ? SCOPF_OK : status;
}

}  // namespace scopf

// ---------------------------------------------------------------------------
// One Newton step at a given iterate (no state update): the unit of work
// of the interior-point inner loop, exposed for benchmarking and tests.
extern "C" int scopf_newton_step(scopf_handle *h, const scopf_state *it, const double *lam_n,
                                 const double *nu0_n, double rho, double mu, double dw_last,
                                 scopf_state *dir, double out[6], int32_t inertia[3]) {
    using namespace scopf;
    if (!h || h->host_only || !it || !lam_n || (h->M.p && !nu0_n) || !(rho > 0) || !(mu > 0))
        return SCOPF_ERR_INVALID_ARG;
    const Model &M = h->M;
    const int64_t n = M.n, m = M.m, p = M.p;
    cudaStream_t s = h->stream;
    if (m) cudaMemcpyAsync(h->lam_n, lam_n, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
    if (p) cudaMemcpyAsync(h->nu0_n, nu0_n, sizeof(double) * p, cudaMemcpyDeviceToDevice, s);
    Ipm I(h);
    const long long apply0 = h->n_refine + h->n_solve_calls;
    const scopf_state &st = *it;
    scopf_state &d = dir ? *dir : h->dir;
    int r = assemble_impl(h, &st, h->lam_n, h->nu0_n, rho, mu, 0.0, h->rhs);
    if (r != SCOPF_OK) return r;
    double delta = 0.0, dwl = dw_last;
    int tries = 0;
    r = I.direction(dwl, delta, tries);
    if (r != SCOPF_OK) return r;
    h->timer.begin(PH_IPM, s);
    note_launch(), k_split<<<nb(M.n_kkt), kT, 0, s>>>(M.n_kkt, h->dm.row_kind, h->dm.row_index, h->sol, d.w,
                                       d.lam, d.yc);
    note_launch(), k_recover<<<nb(n + m + p), kT, 0, s>>>(I.D, st.w, st.r, st.t, st.s, st.lam, st.yc, st.zl,
                                           st.zu, st.zs, h->lam_n, h->nu0_n, rho, mu, d.w, d.lam,
                                           d.yc, d.r, d.t, d.s, d.zl, d.zu, d.zs);
    const double tau = std::fmax(h->opt.tau_min, 1.0 - mu);
    note_launch(), k_ftb<<<kB, kT, 0, s>>>(I.D, st.w, st.s, st.zl, st.zu, st.zs, d.w, d.s, d.zl, d.zu, d.zs, tau,
                            I.dpart);
    // step lengths reduced on the device; the trial point and its filter
    // values follow without a round trip, and the step lengths come back with
    // the trial's partial sums
    double *d_alpha = I.dpart + (size_t)kB * (kPartSlots - 1);
    note_launch(), k_ftb_finish<<<1, kT, 0, s>>>(I.dpart, kB, d_alpha);
    double alpha[2] = {1.0, 1.0};
    cudaMemcpyAsync(alpha, d_alpha, sizeof(alpha), cudaMemcpyDeviceToHost, s);
    I.step(h->trial, st, d, 1.0, 1.0, d_alpha);
    double tht, pht;
    I.trial_eval(h->trial, rho, mu, tht, pht);
    const double ap = alpha[0], az = alpha[1];
    h->timer.end(PH_IPM, s);
    host_sync(h, s);
    h->timer.collect();
    if (out) {
        out[0] = ap;
        out[1] = az;
        out[2] = tht;
        out[3] = pht;
        out[4] = delta;
        out[5] = (double)(h->n_refine + h->n_solve_calls - apply0);
    }
    if (inertia) {
        inertia[0] = (int32_t)n;
        inertia[1] = (int32_t)(m + p);
        inertia[2] = tries;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return SCOPF_ERR_CUDA;
    }
    return SCOPF_OK;
}

extern "C" int scopf_history(scopf_handle *h, int32_t which, int64_t capacity, double *out,
                             int64_t *n_records, int32_t *record_len) {
    using namespace scopf;
    if (!h || (which != 0 && which != 1) || !n_records || !record_len || capacity < 0)
        return SCOPF_ERR_INVALID_ARG;
    const std::vector<double> &v = which == 0 ? h->hist_inner : h->hist_outer;
    const int len = which == 0 ? kHistInner : kHistOuter;
    const int64_t n = (int64_t)v.size() / len;
    *n_records = n;
    *record_len = len;
    if (out) {
        const int64_t k = n < capacity ? n : capacity;
        std::copy(v.begin(), v.begin() + k * len, out);
    }
    return SCOPF_OK;
}

// Continue the NCL method from the handle's current iterate and parameters:
// the end of a previous solve on this handle, or a checkpoint restored with
// scopf_load_state + scopf_set_ncl_params.
extern "C" int ncl_resume(scopf_handle *h, scopf_result *res) {
    using namespace scopf;
    if (!h || h->host_only || !res || !h->have_ncl) return SCOPF_ERR_INVALID_ARG;
    return ncl_solve_impl(h, nullptr, res, true);
}
