/*
 * Oracle sparse LDL^T without pivoting (test infrastructure only).
 *
 * K = L D L' with L unit lower triangular and D diagonal: the pivot-free
 * ("signed Cholesky") factorisation that the NCL regularisation makes
 * possible (Section IV-B).  Plain up-looking algorithm: row k of L solves
 * the sparse triangular system L(0:k,0:k) D y = K(0:k,k), whose nonzero
 * pattern is the set of elimination-tree paths from the nonzeros of
 * K(0:k,k) towards k.  No supernodes, no blocking, one scalar at a time.
 *
 * Input: the upper triangle of the (already permuted) symmetric matrix,
 * stored by columns (Ap, Ai, Ax), row indices sorted ascending.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* Elimination tree (parent) and the number of off-diagonal entries in each
 * column of L (Lnz).  Returns 0. */
int64_t oracle_ldlt_symbolic(int64_t n, const int64_t *Ap, const int64_t *Ai,
                             int64_t *parent, int64_t *Lnz) {
    int64_t *flag = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) {
        parent[k] = -1;
        flag[k] = k;
        Lnz[k] = 0;
        for (int64_t p = Ap[k]; p < Ap[k + 1]; p++) {
            int64_t i = Ai[p];
            if (i >= k) continue;
            /* walk up the tree from i until a node already marked for row k */
            while (flag[i] != k) {
                if (parent[i] == -1) parent[i] = k;
                Lnz[i]++;          /* L(k, i) is structurally nonzero */
                flag[i] = k;
                i = parent[i];
            }
        }
    }
    free(flag);
    return 0;
}

/* Numeric factorisation.  Lp must hold the column pointers from Lnz.
 * Returns the number of pivots with |d| <= pivot_tol. */
int64_t oracle_ldlt_numeric(int64_t n, const int64_t *Ap, const int64_t *Ai,
                            const double *Ax, const int64_t *parent,
                            const int64_t *Lp, int64_t *Li, double *Lx,
                            double *D, double pivot_tol) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *y = (double *)calloc(nn, sizeof(double));
    int64_t *flag = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *pattern = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *fill = (int64_t *)calloc(nn, sizeof(int64_t));
    int64_t nsmall = 0;
    for (int64_t k = 0; k < n; k++) {
        int64_t top = n;
        flag[k] = k;
        for (int64_t p = Ap[k]; p < Ap[k + 1]; p++) {
            int64_t i = Ai[p];
            if (i > k) continue;
            y[i] += Ax[p];
            int64_t len = 0;
            for (; flag[i] != k; i = parent[i]) {
                pattern[len++] = i;
                flag[i] = k;
            }
            while (len > 0) pattern[--top] = pattern[--len];
        }
        double d = y[k];
        y[k] = 0.0;
        for (; top < n; top++) {
            int64_t i = pattern[top];
            double yi = y[i];
            y[i] = 0.0;
            for (int64_t p = Lp[i]; p < Lp[i] + fill[i]; p++) y[Li[p]] -= Lx[p] * yi;
            double lki = yi / D[i];
            d -= lki * yi;
            Li[Lp[i] + fill[i]] = k;
            Lx[Lp[i] + fill[i]] = lki;
            fill[i]++;
        }
        D[k] = d;
        if (fabs(d) <= pivot_tol) nsmall++;
    }
    free(y);
    free(flag);
    free(pattern);
    free(fill);
    return nsmall;
}

/* x <- (L D L')^{-1} x */
void oracle_ldlt_solve(int64_t n, const int64_t *Lp, const int64_t *Li,
                       const double *Lx, const double *D, double *x) {
    for (int64_t j = 0; j < n; j++)
        for (int64_t p = Lp[j]; p < Lp[j + 1]; p++) x[Li[p]] -= Lx[p] * x[j];
    for (int64_t j = 0; j < n; j++) x[j] /= D[j];
    for (int64_t j = n - 1; j >= 0; j--)
        for (int64_t p = Lp[j]; p < Lp[j + 1]; p++) x[j] -= Lx[p] * x[Li[p]];
}
