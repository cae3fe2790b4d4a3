/*
 * CPU oracle for the SVT hot path: plain, slow, float64 C.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package smoke check and the bench's CPU-baseline leg may load this
 * library.  It shares no code, header or constant table with the CUDA path.
 *
 * Contents
 *   oracle_jacobi_svd   dense SVD by one-sided (Hestenes) Jacobi rotations, the textbook
 *                       method (Hestenes 1958; Demmel & Veselic 1992).  It serves the shrink
 *                       operator D_tau of Sec. 2.1, eq. (2.2), which is defined through the SVD.
 *   oracle_splitmix64   the SplitMix64 generator (Steele, Lea & Flood 2014), written from its
 *                       published definition: state += 0x9e3779b97f4a7c15, then two
 *                       xor-shift-multiply rounds and a final xor-shift.
 *   oracle_sample_omega the random-keys sampler of Omega: the m linear ids i*n2+j with the
 *                       smallest (key, id), key = SplitMix64 output number id+1 for the given
 *                       seed.  Every m-subset is equally likely, as Sec. 5.2.1 requires.
 *
 * Compiled with -O2 -ffp-contract=off so that every product and sum rounds separately.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------------------- */
/* One-sided Jacobi SVD                                                                      */
/* ---------------------------------------------------------------------------------------- */

/* Column-major work matrix W (rows x cols); rotate columns p and q by (c, s). */
static void rotate_cols(double *W, int rows, int p, int q, double c, double s) {
    double *wp = W + (size_t)p * rows, *wq = W + (size_t)q * rows;
    for (int i = 0; i < rows; ++i) {
        double a = wp[i], b = wq[i];
        wp[i] = c * a - s * b;
        wq[i] = s * a + c * b;
    }
}

/*
 * SVD of the row-major m x n matrix A:  A = U diag(s) V^T with k = min(m, n) triplets,
 * singular values sorted in decreasing order.
 *   U: m x k row-major, s: k, V: n x k row-major.  Any output pointer may be NULL.
 * Method: orthogonalise the columns of G (G = A if m >= n, else A^T) by plane rotations
 * G <- G J(p,q) chosen so that columns p and q become orthogonal, accumulating the
 * rotations in Q; sweep over all pairs until every pair satisfies
 * |g_p . g_q| <= tol * ||g_p|| ||g_q||.  Then G = U' Sigma with U' orthonormal, G = U' Sigma Q^T.
 * Returns the number of sweeps, or -1 if max_sweeps was exhausted, -2 on allocation failure.
 */
int oracle_jacobi_svd(int m, int n, const double *A, double *U, double *s, double *V, double tol,
                      int max_sweeps) {
    int trans = m < n;
    int rows = trans ? n : m;  /* length of each column of G */
    int cols = trans ? m : n;  /* number of columns of G */
    int k = cols;
    double *G = (double *)malloc(sizeof(double) * (size_t)rows * cols);
    double *Q = (double *)malloc(sizeof(double) * (size_t)cols * cols);
    double *nrm = (double *)malloc(sizeof(double) * (size_t)cols);
    int *ord = (int *)malloc(sizeof(int) * (size_t)cols);
    if (!G || !Q || !nrm || !ord) {
        free(G); free(Q); free(nrm); free(ord);
        return -2;
    }
    /* G column c, entry i:  A[i][c] (no transpose) or A[c][i] (transpose). */
    for (int c = 0; c < cols; ++c)
        for (int i = 0; i < rows; ++i)
            G[(size_t)c * rows + i] = trans ? A[(size_t)c * n + i] : A[(size_t)i * n + c];
    memset(Q, 0, sizeof(double) * (size_t)cols * cols);
    for (int c = 0; c < cols; ++c) Q[(size_t)c * cols + c] = 1.0;

    int sweep = 0, converged = 0;
    while (!converged && sweep < max_sweeps) {
        converged = 1;
        ++sweep;
        for (int p = 0; p < cols - 1; ++p) {
            for (int q = p + 1; q < cols; ++q) {
                const double *gp = G + (size_t)p * rows, *gq = G + (size_t)q * rows;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < rows; ++i) {
                    alpha += gp[i] * gp[i];
                    beta += gq[i] * gq[i];
                    gamma += gp[i] * gq[i];
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
                converged = 0;
                /* Rotation angle that zeroes the (p,q) entry of G^T G:
                   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)). */
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                rotate_cols(G, rows, p, q, c, sn);
                rotate_cols(Q, cols, p, q, c, sn);
            }
        }
    }
    /* Singular values are the column norms; sort decreasing (stable on ties by index). */
    for (int c = 0; c < cols; ++c) {
        double acc = 0.0;
        const double *gc = G + (size_t)c * rows;
        for (int i = 0; i < rows; ++i) acc += gc[i] * gc[i];
        nrm[c] = sqrt(acc);
        ord[c] = c;
    }
    for (int a = 1; a < cols; ++a) {  /* insertion sort */
        int v = ord[a], b = a - 1;
        while (b >= 0 && nrm[ord[b]] < nrm[v]) { ord[b + 1] = ord[b]; --b; }
        ord[b + 1] = v;
    }
    /* G = U' Sigma, A (or A^T) = G Q^T.  Without transpose: U = U', V = Q.  With transpose:
       A^T = U' Sigma Q^T  =>  A = Q Sigma U'^T, so U = Q and V = U'. */
    for (int jj = 0; jj < k; ++jj) {
        int c = ord[jj];
        double sig = nrm[c];
        if (s) s[jj] = sig;
        const double *gc = G + (size_t)c * rows;
        const double *qc = Q + (size_t)c * cols;
        double *left = trans ? V : U;   /* receives U' columns (length rows) */
        double *right = trans ? U : V;  /* receives Q columns (length cols) */
        int ld_left = k, ld_right = k;
        if (left)
            for (int i = 0; i < rows; ++i)
                left[(size_t)i * ld_left + jj] = sig > 0.0 ? gc[i] / sig : 0.0;
        if (right)
            for (int i = 0; i < cols; ++i) right[(size_t)i * ld_right + jj] = qc[i];
    }
    free(G); free(Q); free(nrm); free(ord);
    return converged ? sweep : -1;
}

/* ---------------------------------------------------------------------------------------- */
/* SplitMix64 and the random-keys sampler of Omega                                           */
/* ---------------------------------------------------------------------------------------- */

/* Output number `index` (1-based) of SplitMix64 started from state `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t index) {
    uint64_t z = seed + index * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t key; uint64_t id; } keyed_id;

static int keyed_less(const keyed_id *a, const keyed_id *b) {
    return a->key < b->key || (a->key == b->key && a->id < b->id);
}

/* Max-heap on (key, id): heap[0] is the largest of the m smallest seen so far. */
static void sift_down(keyed_id *h, int64_t n, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, big = i;
        if (l < n && keyed_less(&h[big], &h[l])) big = l;
        if (r < n && keyed_less(&h[big], &h[r])) big = r;
        if (big == i) return;
        keyed_id t = h[i]; h[i] = h[big]; h[big] = t;
        i = big;
    }
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/*
 * Omega = the m ids in [0, n1*n2) with the smallest (key(id), id), key(id) = splitmix64(seed,
 * id + 1).  Written out sorted by id as (rows, cols) = (id / n2, id % n2).
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_sample_omega(int64_t n1, int64_t n2, int64_t m, uint64_t seed, int32_t *rows, int32_t *cols) {
    if (n1 <= 0 || n2 <= 0 || m < 0 || m > n1 * n2) return -1;
    if (m == 0) return 0;
    keyed_id *heap = (keyed_id *)malloc(sizeof(keyed_id) * (size_t)m);
    if (!heap) return -2;
    int64_t N = n1 * n2;
    for (int64_t id = 0; id < m; ++id) {
        heap[id].key = oracle_splitmix64(seed, (uint64_t)id + 1);
        heap[id].id = (uint64_t)id;
    }
    for (int64_t i = m / 2 - 1; i >= 0; --i) sift_down(heap, m, i);
    for (int64_t id = m; id < N; ++id) {
        keyed_id c = {oracle_splitmix64(seed, (uint64_t)id + 1), (uint64_t)id};
        if (keyed_less(&c, &heap[0])) {
            heap[0] = c;
            sift_down(heap, m, 0);
        }
    }
    uint64_t *ids = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
    if (!ids) { free(heap); return -2; }
    for (int64_t i = 0; i < m; ++i) ids[i] = heap[i].id;
    free(heap);
    qsort(ids, (size_t)m, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i < m; ++i) {
        rows[i] = (int32_t)(ids[i] / (uint64_t)n2);
        cols[i] = (int32_t)(ids[i] % (uint64_t)n2);
    }
    free(ids);
    return 0;
}
