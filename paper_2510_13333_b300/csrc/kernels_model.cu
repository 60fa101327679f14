// Model evaluation and KKT assembly kernels (FP64).
//
// Branch elements evaluate the pi-model arc flows of one in-service branch in
// one scenario (Section II, eq. scopf; flows in the textbook polar form),
// their first derivatives and the multiplier-weighted second derivatives
// that enter H = grad^2 (phi + lam' c) of eq. (newtonsystem).  Every element
// writes only its own slots of the value buffer (structure of arrays, so a
// warp's stores are coalesced); the assembly kernel then forms each stored
// KKT entry as a fixed-order sum of its contributions, which keeps the
// result deterministic without atomics.
#include <cmath>

#include "internal.h"
#include "kernels.h"

namespace scopf {

namespace {

constexpr int kThreads = 256;

inline int nblocks(int64_t n, int t = kThreads) {
    int64_t b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : (b > 2147483647 ? 2147483647 : b));
}

// Arc flow F = A vi^2 + B vj^2 + vi vj (al cos th + be sin th), th = th_i - th_j.
__global__ void k_branch(int64_t n_be, const int32_t *__restrict__ bx,
                         const int32_t *__restrict__ blam, const int32_t *__restrict__ bth,
                         const double *__restrict__ par, const double *__restrict__ w,
                         const double *__restrict__ lam, double *__restrict__ ev, int mode) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_be) return;
    const int32_t x0 = bx[4 * e], x1 = bx[4 * e + 1], x2 = bx[4 * e + 2], x3 = bx[4 * e + 3];
    const double thi = x0 >= 0 ? w[x0] : 0.0;
    const double thj = x1 >= 0 ? w[x1] : 0.0;
    const double vi = w[x2], vj = w[x3];
    const double g = par[4 * e], b = par[4 * e + 1], bc = par[4 * e + 2], ir2 = par[4 * e + 3];
    double sn, cs;
    sincos(thi - thj, &sn, &cs);
    const double sh = -(b + 0.5 * bc);
    const double A[4] = {g, sh, 0.0, 0.0};
    const double Bq[4] = {0.0, 0.0, g, sh};
    const double al[4] = {-g, b, -g, b};
    const double be[4] = {-b, -g, b, g};
    double F[4], T[4], Tp[4];
    const double vv = vi * vj;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        T[a] = al[a] * cs + be[a] * sn;
        Tp[a] = -al[a] * sn + be[a] * cs;
        F[a] = A[a] * vi * vi + Bq[a] * vj * vj + vv * T[a];
        ev[(int64_t)(BS_F + a) * n_be + e] = F[a];
    }
    const double hf = (F[0] * F[0] + F[1] * F[1]) * ir2;
    const double ht = (F[2] * F[2] + F[3] * F[3]) * ir2;
    ev[(int64_t)(BS_H + 0) * n_be + e] = hf;
    ev[(int64_t)(BS_H + 1) * n_be + e] = ht;
    if (mode == 0) return;
    double G[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        G[a][0] = vv * Tp[a];
        G[a][1] = -vv * Tp[a];
        G[a][2] = 2.0 * A[a] * vi + vj * T[a];
        G[a][3] = 2.0 * Bq[a] * vj + vi * T[a];
#pragma unroll
        for (int j = 0; j < 4; j++) ev[(int64_t)(BS_DF + 4 * a + j) * n_be + e] = G[a][j];
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        ev[(int64_t)(BS_DH + j) * n_be + e] = 2.0 * ir2 * (F[0] * G[0][j] + F[1] * G[1][j]);
        ev[(int64_t)(BS_DH + 4 + j) * n_be + e] = 2.0 * ir2 * (F[2] * G[2][j] + F[3] * G[3][j]);
    }
    // weights: balance rows carry -F; thermal rows carry (p^2 + q^2) ir2
    double wt[4];
#pragma unroll
    for (int a = 0; a < 4; a++) wt[a] = -lam[blam[4 * e + a]];
    const int32_t t0 = bth[2 * e], t1 = bth[2 * e + 1];
    const double mu0 = t0 >= 0 ? 2.0 * ir2 * lam[t0] : 0.0;
    const double mu1 = t1 >= 0 ? 2.0 * ir2 * lam[t1] : 0.0;
    // effective weight of each flow's own Hessian: -lam_a + mu_e * F_a
    const double we[4] = {wt[0] + mu0 * F[0], wt[1] + mu0 * F[1], wt[2] + mu1 * F[2],
                          wt[3] + mu1 * F[3]};
    // sum_a we_a * Hess(F_a)
    double sT = 0, sTp = 0, sA = 0, sB = 0;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        sT += we[a] * T[a];
        sTp += we[a] * Tp[a];
        sA += we[a] * A[a];
        sB += we[a] * Bq[a];
    }
    // Hess(F) entries (upper triangle, x = th_i, th_j, v_i, v_j), T'' = -T
    double H[10];
    H[0] = -vv * sT;        // (0,0)
    H[1] = vv * sT;         // (0,1)
    H[2] = vj * sTp;        // (0,2)
    H[3] = vi * sTp;        // (0,3)
    H[4] = -vv * sT;        // (1,1)
    H[5] = -vj * sTp;       // (1,2)
    H[6] = -vi * sTp;       // (1,3)
    H[7] = 2.0 * sA;        // (2,2)
    H[8] = sT;              // (2,3)
    H[9] = 2.0 * sB;        // (3,3)
    // Gauss-Newton part of the thermal rows: mu_e (grad p grad p' + grad q grad q')
    int h = 0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = i; j < 4; j++, h++)
            H[h] += mu0 * (G[0][i] * G[0][j] + G[1][i] * G[1][j]) +
                    mu1 * (G[2][i] * G[2][j] + G[3][i] * G[3][j]);
#pragma unroll
    for (int q = 0; q < 10; q++) ev[(int64_t)(BS_HESS + q) * n_be + e] = H[q];
}

__global__ void k_shunt(int64_t n_se, const int32_t *__restrict__ sv, const int32_t *__restrict__ sP,
                        const int32_t *__restrict__ sQ, const double *__restrict__ G,
                        const double *__restrict__ Bs, const double *__restrict__ w,
                        const double *__restrict__ lam, double *__restrict__ ev, int mode) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_se) return;
    const double v = w[sv[e]];
    ev[0 * n_se + e] = -G[e] * v * v;
    ev[1 * n_se + e] = Bs[e] * v * v;
    if (mode == 0) return;
    ev[2 * n_se + e] = -2.0 * G[e] * v;
    ev[3 * n_se + e] = 2.0 * Bs[e] * v;
    ev[4 * n_se + e] = -2.0 * G[e] * lam[sP[e]] + 2.0 * Bs[e] * lam[sQ[e]];
}

__global__ void k_comp(int64_t p, const int64_t *__restrict__ c1, const int64_t *__restrict__ c2,
                       const double *__restrict__ w, const double *__restrict__ yc,
                       double *__restrict__ ev) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= p) return;
    ev[q] = w[c2[q]];
    ev[p + q] = w[c1[q]];
    ev[2 * p + q] = yc[q];
}

__global__ void k_cons(int64_t m, const double *__restrict__ cc, const int64_t *__restrict__ ptr,
                       const int64_t *__restrict__ idx, const double *__restrict__ coef,
                       const double *__restrict__ ev, const double *__restrict__ w,
                       double *__restrict__ c) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double v = cc[r];
    for (int64_t k = ptr[r]; k < ptr[r + 1]; k++) {
        int64_t s = idx[k];
        v += coef[k] * (s >= 0 ? ev[s] : w[-s - 1]);
    }
    c[r] = v;
}

__global__ void k_grad(int ng, int64_t border0, const double *__restrict__ c2,
                       const double *__restrict__ c1, const double *__restrict__ w,
                       double *__restrict__ g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    // d/dp [c2 (100 p)^2 + c1 (100 p)] / 1e4
    const double p = w[border0 + i] * 100.0;
    g[border0 + i] = (2.0 * c2[i] * p + c1[i]) * 100.0 / 1.0e4;
}

__global__ void k_diag(int64_t n_kkt, const int8_t *__restrict__ kind,
                       const int64_t *__restrict__ index, const double *__restrict__ wl,
                       const double *__restrict__ wu, const double *__restrict__ w,
                       const double *__restrict__ zl, const double *__restrict__ zu,
                       const double *__restrict__ sv, const double *__restrict__ zs, DScalar rho_,
                       DScalar delta_w_, double *__restrict__ diag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_kkt) return;
    const double rho = rho_.get(), delta_w = delta_w_.get();
    const int8_t k = kind[i];
    const int64_t j = index[i];
    double d;
    if (k == 0) {
        d = delta_w;
        const double l = wl[j], u = wu[j], x = w[j];
        if (l > -INFINITY) d += zl[j] / (x - l);
        if (u < INFINITY) d += zu[j] / (u - x);
    } else if (k == 1) {
        d = -1.0 / rho;
    } else {
        d = -(1.0 / rho + sv[j] / zs[j]);
    }
    diag[i] = d;
}

__global__ void k_assemble(int64_t nnz, const int32_t *__restrict__ row,
                           const int32_t *__restrict__ col, const int64_t *__restrict__ cptr,
                           const int64_t *__restrict__ src, const double *__restrict__ coef,
                           const double *__restrict__ ev, const double *__restrict__ diag,
                           double *__restrict__ kval) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnz) return;
    double v = 0.0;
    for (int64_t q = cptr[j]; q < cptr[j + 1]; q++) {
        const int64_t s = src[q];
        v += coef[q] * (s >= 0 ? ev[s] : 1.0);
    }
    const int64_t r = row[j];
    if (col[j] == r) v += diag[r];
    kval[j] = v;
}

__device__ __forceinline__ double dual_term(int64_t q, const int32_t *__restrict__ col,
                                            const int8_t *__restrict__ kind,
                                            const int64_t *__restrict__ index,
                                            const double *__restrict__ kval,
                                            const double *__restrict__ lam,
                                            const double *__restrict__ yc) {
    const int64_t c = col[q];
    const int8_t k = kind[c];
    if (k == 1) return kval[q] * lam[index[c]];
    if (k == 2) return kval[q] * yc[index[c]];
    return 0.0;
}

__global__ void k_dual_product(int64_t n_kkt, const int64_t *__restrict__ ptr,
                               const int32_t *__restrict__ col, const int8_t *__restrict__ kind,
                               const int64_t *__restrict__ index, const double *__restrict__ kval,
                               const double *__restrict__ g, const double *__restrict__ lam,
                               const double *__restrict__ yc, double *__restrict__ gw,
                               const int8_t *__restrict__ is_long) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_kkt || kind[i] != 0 || is_long[i]) return;
    double s = 0.0;
    for (int64_t q = ptr[i]; q < ptr[i + 1]; q++) s += dual_term(q, col, kind, index, kval, lam, yc);
    const int64_t wi = index[i];
    gw[wi] = g[wi] + s;
}

// the same for the long rows, one warp per row
__global__ void k_dual_product_long(int64_t n_long, const int64_t *__restrict__ rows,
                                    const int64_t *__restrict__ ptr,
                                    const int32_t *__restrict__ col,
                                    const int8_t *__restrict__ kind,
                                    const int64_t *__restrict__ index,
                                    const double *__restrict__ kval, const double *__restrict__ g,
                                    const double *__restrict__ lam, const double *__restrict__ yc,
                                    double *__restrict__ gw) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_long) return;
    const int64_t i = rows[w];
    if (kind[i] != 0) return;
    double s = 0.0;
    for (int64_t q = ptr[i] + lane; q < ptr[i + 1]; q += 32)
        s += dual_term(q, col, kind, index, kval, lam, yc);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int64_t wi = index[i];
        gw[wi] = g[wi] + s;
    }
}

__global__ void k_rhs(int64_t n_kkt, const int8_t *__restrict__ kind,
                      const int64_t *__restrict__ index, const double *__restrict__ wl,
                      const double *__restrict__ wu, const int64_t *__restrict__ c1,
                      const int64_t *__restrict__ c2, RhsArgs a, double *__restrict__ rhs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_kkt) return;
    const double mu = a.mu.get(), rho = a.rho.get();
    const int8_t k = kind[i];
    const int64_t j = index[i];
    double v;
    if (k == 0) {
        double rw = a.gw[j];
        const double l = wl[j], u = wu[j], x = a.w[j];
        if (l > -INFINITY) rw -= mu / (x - l);
        if (u < INFINITY) rw += mu / (u - x);
        v = -rw;
    } else if (k == 1) {
        v = -(a.c[j] - a.r[j]) - (a.lam_n[j] + rho * a.r[j] - a.lam[j]) / rho;
    } else {
        const double s = a.sv[j];
        const double py = a.w[c1[j]] * a.w[c2[j]] - a.t[j] + s;
        v = -py - (a.nu0_n[j] + rho * a.t[j] - a.yc[j]) / rho -
            (mu / s - a.yc[j]) * s / a.zs[j];
    }
    rhs[i] = v;
}

// y = b - K x (b may be NULL: y = -K x ... used with sign = -1 for y = K x)
__global__ void k_residual(int64_t n_kkt, const int64_t *__restrict__ ptr,
                           const int32_t *__restrict__ col, const double *__restrict__ kval,
                           const double *__restrict__ x, const double *__restrict__ b,
                           double *__restrict__ y, const int8_t *__restrict__ is_long,
                           double sign) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_kkt || is_long[i]) return;
    double s = 0.0;
    for (int64_t q = ptr[i]; q < ptr[i + 1]; q++) s += kval[q] * x[col[q]];
    y[i] = (b ? b[i] : 0.0) + sign * s;
}

__global__ void k_residual_long(int64_t n_long, const int64_t *__restrict__ rows,
                                const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                const double *__restrict__ kval, const double *__restrict__ x,
                                const double *__restrict__ b, double *__restrict__ y,
                                double sign) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_long) return;
    const int64_t i = rows[w];
    double s = 0.0;
    for (int64_t q = ptr[i] + lane; q < ptr[i + 1]; q += 32) s += kval[q] * x[col[q]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = (b ? b[i] : 0.0) + sign * s;
}

template <int OP>
__global__ void k_reduce(const double *__restrict__ x, int64_t n, double *__restrict__ out) {
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fabs(x[i]);
        acc = OP == 0 ? fmax(acc, v) : acc + v;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            sh[threadIdx.x] = OP == 0 ? fmax(sh[threadIdx.x], sh[threadIdx.x + s])
                                      : sh[threadIdx.x] + sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

constexpr int kReduceBlocks = 296;

__global__ void k_axpy(int64_t n, double a, const double *__restrict__ x, double *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

}  // namespace

void launch_axpy(int64_t n, double a, const double *x, double *y, cudaStream_t s) {
    if (n) note_launch(), k_axpy<<<nblocks(n), kThreads, 0, s>>>(n, a, x, y);
}

namespace {

__global__ void k_multi_dot(const double *__restrict__ V, int64_t n, int k,
                            const double *__restrict__ w, double *__restrict__ partial) {
    __shared__ double sh[kThreads];
    for (int j = 0; j < k; j++) {
        const double *v = V + (int64_t)j * n;
        double acc = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            acc += v[i] * w[i];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + j] = sh[0];
        __syncthreads();
    }
}

struct Coefs {
    double c[kMaxKrylov];
};

__global__ void k_multi_axpy(double *__restrict__ w, const double *__restrict__ V, int64_t n,
                             int k, Coefs cf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int j = 0; j < k; j++) acc -= cf.c[j] * V[(int64_t)j * n + i];
    w[i] = acc;
}

__global__ void k_scale_copy(int64_t n, double a, const double *__restrict__ x,
                             double *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

// one warp per column: lanes stride over the partials, then a fixed-order
// warp reduction
__global__ void k_dot_finish(const double *__restrict__ partial, int k, double *__restrict__ out,
                             int take_sqrt) {
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= k) return;
    double a = 0.0;
    for (int b = lane; b < kDotBlocks; b += 32) a += partial[(int64_t)b * k + j];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[j] = take_sqrt ? sqrt(fmax(a, 0.0)) : a;
}

__global__ void k_multi_axpy_dev(double *__restrict__ w, const double *__restrict__ V, int64_t n,
                                 int k, const double *__restrict__ c, double sign) {
    __shared__ double cs[kMaxKrylov];
    if (threadIdx.x < k) cs[threadIdx.x] = sign * c[threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int j = 0; j < k; j++) acc -= cs[j] * V[(int64_t)j * n + i];
    w[i] = acc;
}

__global__ void k_scale_inv(int64_t n, const double *__restrict__ den, const double *__restrict__ x,
                            double *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = *den;
    y[i] = d != 0.0 ? x[i] / d : 0.0;
}

__global__ void k_gmres_init(double *st, GmresLayout L) {
    for (int i = threadIdx.x; i <= L.m; i += blockDim.x) st[L.g + i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) st[L.g] = st[L.sc + 0];
}

// Givens rotations on the Hessenberg column (Saad, Iterative Methods for
// Sparse Linear Systems, Alg. 6.9 with the flexible variant of Alg. 9.6)
__global__ void k_gmres_column(double *st, GmresLayout L, int j) {
    if (threadIdx.x != 0) return;
    double *H = st + L.H;
    const int ld = L.m + 1;
    double *col = H + (int64_t)j * ld;
    for (int i = 0; i <= j; i++) col[i] = st[L.c1 + i] + st[L.c2 + i];
    col[j + 1] = st[L.sc + 1];
    double *cs = st + L.cs, *sn = st + L.sn, *g = st + L.g;
    for (int i = 0; i < j; i++) {
        const double a = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = a;
    }
    const double den = hypot(col[j], col[j + 1]);
    cs[j] = den > 0.0 ? col[j] / den : 1.0;
    sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    st[L.sc + 2] = fabs(g[j + 1]);
}

__global__ void k_gmres_solve(double *st, GmresLayout L, int k) {
    if (threadIdx.x != 0) return;
    const double *H = st + L.H;
    const int ld = L.m + 1;
    double y[kMaxKrylov];
    for (int i = k - 1; i >= 0; i--) {
        double a = st[L.g + i];
        for (int q = i + 1; q < k; q++) a -= H[(int64_t)q * ld + i] * y[q];
        const double d = H[(int64_t)i * ld + i];
        y[i] = d != 0.0 ? a / d : 0.0;
    }
    for (int i = 0; i < k; i++) st[L.c1 + i] = -y[i];
}

__global__ void k_diag_gather(int64_t n, const int64_t *__restrict__ pos,
                              const double *__restrict__ kval, double *__restrict__ base) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) base[i] = kval[pos[i]];
}

__global__ void k_diag_set(int64_t n, const int64_t *__restrict__ pos,
                           const double *__restrict__ base, double shift,
                           double *__restrict__ kval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) kval[pos[i]] = base[i] + shift;
}

// count the listed primal rows whose diagonal entry is exactly zero
__global__ void k_count_zero_diag(int64_t n, const int64_t *__restrict__ idx,
                                  const double *__restrict__ base, int *__restrict__ count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool z = i < n && base[idx[i]] == 0.0;
    const unsigned b = __ballot_sync(0xffffffffu, z);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));
}

}  // namespace

void launch_count_zero_diag(int64_t n, const int64_t *idx, const double *base, int *count,
                            cudaStream_t s) {
    cudaMemsetAsync(count, 0, sizeof(int), s);
    if (n) note_launch(), k_count_zero_diag<<<nblocks(n), kThreads, 0, s>>>(n, idx, base, count);
}

void launch_diag_gather(int64_t n, const int64_t *pos, const double *kval, double *base,
                        cudaStream_t s) {
    if (n) note_launch(), k_diag_gather<<<nblocks(n), kThreads, 0, s>>>(n, pos, kval, base);
}

void launch_diag_set(int64_t n, const int64_t *pos, const double *base, double shift,
                     double *kval, cudaStream_t s) {
    if (n) note_launch(), k_diag_set<<<nblocks(n), kThreads, 0, s>>>(n, pos, base, shift, kval);
}

GmresLayout gmres_layout(int m) {
    GmresLayout L;
    L.m = m;
    L.H = 0;
    L.cs = L.H + (m + 1) * m;
    L.sn = L.cs + m;
    L.g = L.sn + m;
    L.c1 = L.g + m + 1;
    L.c2 = L.c1 + kMaxKrylov;
    L.sc = L.c2 + kMaxKrylov;
    L.total = L.sc + 8;
    return L;
}

// ---- device-resident Krylov loop (kernels of a CUDA graph whose WHILE node
// repeats one Krylov step): the column j and the counts come from KrylovCtl
// in device memory, so one captured step serves every j.
namespace {

__global__ void k_kry_start(KrylovCtl *c, int it, int max_it, double target) {
    c->j = 0;
    c->it = it;
    c->max_it = max_it;
    c->jend = 0;
    c->target = target;
}

// out = V_j (the current basis vector, into the preconditioner's input)
__global__ void k_kry_gather(int64_t n, const double *__restrict__ V, const KrylovCtl *__restrict__ c,
                             double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = V[(int64_t)c->j * n + i];
}

// Z_j = in (the preconditioned vector, kept for the solution update)
__global__ void k_kry_scatter(int64_t n, const double *__restrict__ in, double *__restrict__ Z,
                              const KrylovCtl *__restrict__ c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Z[(int64_t)c->j * n + i] = in[i];
}

// partial dot products of V_0 .. V_j with w (k = j + 1 from the device)
__global__ void k_kry_multi_dot(const double *__restrict__ V, int64_t n,
                                const KrylovCtl *__restrict__ c, const double *__restrict__ w,
                                double *__restrict__ partial) {
    __shared__ double sh[kThreads];
    const int k = c->j + 1;
    for (int j = 0; j < k; j++) {
        const double *v = V + (int64_t)j * n;
        double acc = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            acc += v[i] * w[i];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + j] = sh[0];
        __syncthreads();
    }
}

__global__ void k_kry_dot_finish(const double *__restrict__ partial,
                                 const KrylovCtl *__restrict__ c, double *__restrict__ out) {
    const int k = c->j + 1;
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= k) return;
    double a = 0.0;
    for (int b = lane; b < kDotBlocks; b += 32) a += partial[(int64_t)b * k + j];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[j] = a;
}

// w -= sum_{q <= j} coef[q] V_q (kadd = 1), or x -= sum_{q < jend} coef[q] Z_q
// (kadd = 0 with use_jend)
__global__ void k_kry_axpy(double *__restrict__ w, const double *__restrict__ V, int64_t n,
                           const KrylovCtl *__restrict__ c, int use_jend,
                           const double *__restrict__ coef) {
    __shared__ double cs[kMaxKrylov];
    const int k = use_jend ? c->jend : c->j + 1;
    if ((int)threadIdx.x < k) cs[threadIdx.x] = coef[threadIdx.x];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int q = 0; q < k; q++) acc -= cs[q] * V[(int64_t)q * n + i];
    w[i] = acc;
}

// V_{j+1} = w / *den (0 if *den == 0)
__global__ void k_kry_scale_out(int64_t n, const double *__restrict__ den,
                                const double *__restrict__ w, double *__restrict__ V,
                                const KrylovCtl *__restrict__ c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = *den;
    V[(int64_t)(c->j + 1) * n + i] = d != 0.0 ? w[i] / d : 0.0;
}

// column j of the Hessenberg matrix and its Givens rotations (the same
// arithmetic as k_gmres_column), then the loop control: advance j, count the
// preconditioner application, and keep looping while the residual estimate
// is above target, columns remain and the refinement budget is not spent
__global__ void k_kry_column_next(double *st, GmresLayout L, KrylovCtl *c,
                                  cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0) return;
    const int j = c->j;
    double *H = st + L.H;
    const int ld = L.m + 1;
    double *col = H + (int64_t)j * ld;
    for (int i = 0; i <= j; i++) col[i] = st[L.c1 + i] + st[L.c2 + i];
    col[j + 1] = st[L.sc + 1];
    double *cs = st + L.cs, *sn = st + L.sn, *g = st + L.g;
    for (int i = 0; i < j; i++) {
        const double a = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = a;
    }
    const double den = hypot(col[j], col[j + 1]);
    cs[j] = den > 0.0 ? col[j] / den : 1.0;
    sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    st[L.sc + 2] = fabs(g[j + 1]);
    const int jn = j + 1;
    c->j = jn;
    c->jend = jn;
    c->it += 1;
    const bool more = st[L.sc + 2] > c->target && jn < L.m && c->it < c->max_it;
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// small triangular solve for the jend columns of the cycle
__global__ void k_kry_solve(double *st, GmresLayout L, const KrylovCtl *c) {
    if (threadIdx.x != 0) return;
    const int k = c->jend;
    const double *H = st + L.H;
    const int ld = L.m + 1;
    double y[kMaxKrylov];
    for (int i = k - 1; i >= 0; i--) {
        double a = st[L.g + i];
        for (int q = i + 1; q < k; q++) a -= H[(int64_t)q * ld + i] * y[q];
        const double d = H[(int64_t)i * ld + i];
        y[i] = d != 0.0 ? a / d : 0.0;
    }
    for (int i = 0; i < k; i++) st[L.c1 + i] = -y[i];
}

}  // namespace

void launch_kry_start(KrylovCtl *c, int it, int max_it, double target, cudaStream_t s) {
    note_launch(), k_kry_start<<<1, 1, 0, s>>>(c, it, max_it, target);
}
void launch_kry_gather(int64_t n, const double *V, const KrylovCtl *c, double *out, cudaStream_t s) {
    note_launch(), k_kry_gather<<<nblocks(n), kThreads, 0, s>>>(n, V, c, out);
}
void launch_kry_scatter(int64_t n, const double *in, double *Z, const KrylovCtl *c, cudaStream_t s) {
    note_launch(), k_kry_scatter<<<nblocks(n), kThreads, 0, s>>>(n, in, Z, c);
}
void launch_kry_multi_dot(const double *V, int64_t n, const KrylovCtl *c, const double *w,
                          double *partial, cudaStream_t s) {
    note_launch(), k_kry_multi_dot<<<kDotBlocks, kThreads, 0, s>>>(V, n, c, w, partial);
}
void launch_kry_dot_finish(const double *partial, const KrylovCtl *c, double *out, cudaStream_t s) {
    note_launch(), k_kry_dot_finish<<<1, 32 * kMaxKrylov, 0, s>>>(partial, c, out);
}
void launch_kry_axpy(double *w, const double *V, int64_t n, const KrylovCtl *c, bool use_jend,
                     const double *coef, cudaStream_t s) {
    if (n) note_launch(), k_kry_axpy<<<nblocks(n), kThreads, 0, s>>>(w, V, n, c, use_jend ? 1 : 0, coef);
}
void launch_kry_scale_out(int64_t n, const double *den, const double *w, double *V,
                          const KrylovCtl *c, cudaStream_t s) {
    note_launch(), k_kry_scale_out<<<nblocks(n), kThreads, 0, s>>>(n, den, w, V, c);
}
void launch_kry_column_next(double *st, int m, KrylovCtl *c, cudaGraphConditionalHandle loop,
                            cudaStream_t s) {
    note_launch(), k_kry_column_next<<<1, 32, 0, s>>>(st, gmres_layout(m), c, loop);
}
void launch_kry_solve(double *st, int m, const KrylovCtl *c, cudaStream_t s) {
    note_launch(), k_kry_solve<<<1, 32, 0, s>>>(st, gmres_layout(m), c);
}

void launch_dot_finish(const double *partial, int k, double *out, bool take_sqrt, cudaStream_t s) {
    note_launch(), k_dot_finish<<<1, 32 * k, 0, s>>>(partial, k, out, take_sqrt ? 1 : 0);
}

void launch_multi_axpy_dev(double *w, const double *V, int64_t n, int k, const double *c,
                           double sign, cudaStream_t s) {
    if (n) note_launch(), k_multi_axpy_dev<<<nblocks(n), kThreads, 0, s>>>(w, V, n, k, c, sign);
}

void launch_scale_inv(int64_t n, const double *den, const double *x, double *y, cudaStream_t s) {
    if (n) note_launch(), k_scale_inv<<<nblocks(n), kThreads, 0, s>>>(n, den, x, y);
}

void launch_gmres_init(double *st, int m, cudaStream_t s) {
    note_launch(), k_gmres_init<<<1, 64, 0, s>>>(st, gmres_layout(m));
}

void launch_gmres_column(double *st, int m, int j, cudaStream_t s) {
    note_launch(), k_gmres_column<<<1, 32, 0, s>>>(st, gmres_layout(m), j);
}

void launch_gmres_solve(double *st, int m, int k, cudaStream_t s) {
    note_launch(), k_gmres_solve<<<1, 32, 0, s>>>(st, gmres_layout(m), k);
}

void reduce_maxabs2(const double *a, const double *b, int64_t n, double *d_out, double *scratch,
                    cudaStream_t s) {
    note_launch(), k_reduce<0><<<kReduceBlocks, kThreads, 0, s>>>(a, n, scratch);
    note_launch(), k_reduce<0><<<1, kThreads, 0, s>>>(scratch, kReduceBlocks, d_out);
    note_launch(), k_reduce<0><<<kReduceBlocks, kThreads, 0, s>>>(b, n, scratch + kReduceBlocks);
    note_launch(), k_reduce<0><<<1, kThreads, 0, s>>>(scratch + kReduceBlocks, kReduceBlocks, d_out + 1);
}

void launch_multi_dot(const double *V, int64_t n, int k, const double *w, double *partial,
                      cudaStream_t s) {
    note_launch(), k_multi_dot<<<kDotBlocks, kThreads, 0, s>>>(V, n, k, w, partial);
}

void launch_multi_axpy(double *w, const double *V, int64_t n, int k, const double *c,
                       cudaStream_t s) {
    Coefs cf;
    for (int j = 0; j < k && j < kMaxKrylov; j++) cf.c[j] = c[j];
    note_launch(), k_multi_axpy<<<nblocks(n), kThreads, 0, s>>>(w, V, n, k, cf);
}

void launch_scale_copy(int64_t n, double a, const double *x, double *y, cudaStream_t s) {
    if (n) note_launch(), k_scale_copy<<<nblocks(n), kThreads, 0, s>>>(n, a, x, y);
}

void launch_spmv(const DevModel &M, const double *kval, const double *x, double *y,
                 cudaStream_t s) {
    note_launch(), k_residual<<<nblocks(M.n_kkt), kThreads, 0, s>>>(M.n_kkt, M.kkt_ptr, M.kkt_col, kval, x,
                                                     nullptr, y, M.is_long, 1.0);
    if (M.n_long)
        note_launch(), k_residual_long<<<nblocks(32 * M.n_long), kThreads, 0, s>>>(
            M.n_long, M.long_rows, M.kkt_ptr, M.kkt_col, kval, x, nullptr, y, 1.0);
}

void launch_eval_elements(const DevModel &M, const double *w, const double *lam, const double *yc,
                          double *ev, int mode, cudaStream_t s) {
    if (M.n_be)
        note_launch(), k_branch<<<nblocks(M.n_be), kThreads, 0, s>>>(M.n_be, M.be_x, M.be_lam, M.be_th, M.be_par,
                                                      w, lam, ev + M.ev_branch0, mode);
    if (M.n_se)
        note_launch(), k_shunt<<<nblocks(M.n_se), kThreads, 0, s>>>(M.n_se, M.se_v, M.se_P, M.se_Q, M.se_G,
                                                     M.se_B, w, lam, ev + M.ev_shunt0, mode);
    if (M.p && mode)
        note_launch(), k_comp<<<nblocks(M.p), kThreads, 0, s>>>(M.p, M.comp1, M.comp2, w, yc, ev + M.ev_comp0);
}

void launch_constraints(const DevModel &M, const double *w, const double *ev, double *c,
                        cudaStream_t s) {
    if (M.m)
        note_launch(), k_cons<<<nblocks(M.m), kThreads, 0, s>>>(M.m, M.c_const, M.cf_ptr, M.cf_idx, M.cf_coef, ev,
                                                 w, c);
}

void launch_gradient(const DevModel &M, const double *w, double *g, cudaStream_t s) {
    cudaMemsetAsync(g, 0, sizeof(double) * M.n, s);
    note_launch(), k_grad<<<nblocks(M.ng), kThreads, 0, s>>>(M.ng, M.border0, M.c2, M.c1, w, g);
}

void launch_diag_terms(const DevModel &M, const double *w, const double *zl, const double *zu,
                       const double *sv, const double *zs, DScalar rho, DScalar delta_w,
                       double *diag, cudaStream_t s) {
    note_launch(), k_diag<<<nblocks(M.n_kkt), kThreads, 0, s>>>(M.n_kkt, M.row_kind, M.row_index, M.wl, M.wu, w,
                                                 zl, zu, sv, zs, rho, delta_w, diag);
}

void launch_assemble(const DevModel &M, const double *ev, const double *diag, double *kval,
                     cudaStream_t s) {
    note_launch(), k_assemble<<<nblocks(M.nnz), kThreads, 0, s>>>(M.nnz, M.kkt_row, M.kkt_col, M.ctr_ptr,
                                                   M.ctr_src, M.ctr_coef, ev, diag, kval);
}

void launch_dual_product(const DevModel &M, const double *kval, const double *g, const double *lam,
                         const double *yc, double *gw, cudaStream_t s) {
    note_launch(), k_dual_product<<<nblocks(M.n_kkt), kThreads, 0, s>>>(M.n_kkt, M.kkt_ptr, M.kkt_col, M.row_kind,
                                                         M.row_index, kval, g, lam, yc, gw,
                                                         M.is_long);
    if (M.n_long)
        note_launch(), k_dual_product_long<<<nblocks(32 * M.n_long), kThreads, 0, s>>>(
            M.n_long, M.long_rows, M.kkt_ptr, M.kkt_col, M.row_kind, M.row_index, kval, g, lam,
            yc, gw);
}

void launch_rhs(const DevModel &M, const RhsArgs &a, double *rhs, cudaStream_t s) {
    note_launch(), k_rhs<<<nblocks(M.n_kkt), kThreads, 0, s>>>(M.n_kkt, M.row_kind, M.row_index, M.wl, M.wu,
                                                M.comp1, M.comp2, a, rhs);
}

void launch_residual(const DevModel &M, const double *kval, const double *x, const double *b,
                     double *y, cudaStream_t s) {
    note_launch(), k_residual<<<nblocks(M.n_kkt), kThreads, 0, s>>>(M.n_kkt, M.kkt_ptr, M.kkt_col, kval, x, b, y,
                                                     M.is_long, -1.0);
    if (M.n_long)
        note_launch(), k_residual_long<<<nblocks(32 * M.n_long), kThreads, 0, s>>>(
            M.n_long, M.long_rows, M.kkt_ptr, M.kkt_col, kval, x, b, y, -1.0);
}

void reduce_maxabs(const double *x, int64_t n, double *d_out, double *scratch, cudaStream_t s) {
    note_launch(), k_reduce<0><<<kReduceBlocks, kThreads, 0, s>>>(x, n, scratch);
    note_launch(), k_reduce<0><<<1, kThreads, 0, s>>>(scratch, kReduceBlocks, d_out);
}

void reduce_sumabs(const double *x, int64_t n, double *d_out, double *scratch, cudaStream_t s) {
    note_launch(), k_reduce<1><<<kReduceBlocks, kThreads, 0, s>>>(x, n, scratch);
    note_launch(), k_reduce<1><<<1, kThreads, 0, s>>>(scratch, kReduceBlocks, d_out);
}

}  // namespace scopf
