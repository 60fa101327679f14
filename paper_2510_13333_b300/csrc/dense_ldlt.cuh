// Dense LDL^T triangular solves for one CTA (FP64): y <- (L D L')^-1 y with
// L unit lower triangular stored below the diagonal of S (column-major,
// n x n) and D on its diagonal.  Blocks of 32 rows: warp 0 solves each
// 32 x 32 diagonal block with register shuffles, the whole CTA updates the
// remaining rows.  Used for the border (Schur complement) block of
// eq. (newtonsystem).
#pragma once

namespace scopf {

// first: y is zero above this row on entry (the forward sweep starts at its
// 32-row block)
template <int NT>
__device__ void block_ldlt_solve(const double *__restrict__ S, int n, double *__restrict__ y,
                                 int first = 0) {
    __shared__ double blk[32][33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
    for (int b0 = (first / 32) * 32; b0 < n; b0 += 32) {
        const int bs = n - b0 < 32 ? n - b0 : 32;
        for (int t = tid; t < 32 * 32; t += NT) {
            const int c = t >> 5, r = t & 31;
            blk[r][c] = (r < bs && c < bs) ? S[(int64_t)(b0 + c) * n + b0 + r] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            double yl = lane < bs ? y[b0 + lane] : 0.0;
            for (int j = 0; j < bs; j++) {
                const double yj = __shfl_sync(0xffffffffu, yl, j);
                if (lane > j) yl -= blk[lane][j] * yj;
            }
            if (lane < bs) y[b0 + lane] = yl;
        }
        __syncthreads();
        for (int i = b0 + bs + tid; i < n; i += NT) {
            double acc = 0.0;
            for (int j = 0; j < bs; j++) acc += S[(int64_t)(b0 + j) * n + i] * y[b0 + j];
            y[i] -= acc;
        }
        __syncthreads();
    }
    for (int c = tid; c < n; c += NT) y[c] /= S[(int64_t)c * n + c];
    __syncthreads();
    const int nblk = (n + 31) / 32;
    for (int bi = nblk - 1; bi >= 0; bi--) {
        const int b0 = bi * 32, bs = n - b0 < 32 ? n - b0 : 32;
        for (int il = warp; il < bs; il += nw) {
            const int i = b0 + il;
            const double *col = S + (int64_t)i * n;
            double acc = 0.0;
            for (int k = b0 + bs + lane; k < n; k += 32) acc += col[k] * y[k];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) y[i] -= acc;
        }
        for (int t = tid; t < 32 * 32; t += NT) {
            const int c = t >> 5, r = t & 31;
            blk[r][c] = (r < bs && c < bs) ? S[(int64_t)(b0 + c) * n + b0 + r] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            double xl = lane < bs ? y[b0 + lane] : 0.0;
            for (int k = bs - 1; k >= 0; k--) {
                const double xk = __shfl_sync(0xffffffffu, xl, k);
                if (lane < k) xl -= blk[k][lane] * xk;
            }
            if (lane < bs) y[b0 + lane] = xl;
        }
        __syncthreads();
    }
}

}  // namespace scopf
