/*
 * FP64 brute-force exact k-nearest-neighbour search.
 *
 * TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load this library; the
 * CUDA path never does.
 *
 * Definition followed (Sec. 2.1, Eq. for b^2 and the index map I(x, k)):
 * I(x, k) is the k-th closest sample to x, with I(x^(i), 0) = i, so the point
 * itself is excluded and its k nearest *other* samples are returned.
 *
 * Canonical squared distance, evaluated in IEEE FP64 round-to-nearest with no
 * contraction (build with -ffp-contract=off):
 *     delta_r = x_ir - x_jr,  s_r = delta_r * delta_r,
 *     d2 = ((s_0 + s_1) + s_2) + ...   (ascending r)
 * RN subtraction is antisymmetric, so d2(i, j) == d2(j, i) bit for bit.
 * Neighbours are ordered by (d2, j) ascending: distance first, index second.
 * Duplicate points are legal neighbours (d2 = 0).
 */
#include <stdint.h>

static inline double canon_d2(const float* xi, const float* xj, int32_t m)
{
    double acc = 0.0;
    for (int32_t r = 0; r < m; ++r) {
        double dl = (double)xi[r] - (double)xj[r];
        double s = dl * dl;
        acc = (r == 0) ? s : acc + s;
    }
    return acc;
}

/* Squared distances of explicit pairs (a[t], b[t]) in the canonical order. */
void oracle_pair_d2(const float* x, int32_t m, const int64_t* a, const int64_t* b, int64_t npairs, double* out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < npairs; ++t)
        out[t] = canon_d2(x + a[t] * m, x + b[t] * m, m);
}

/*
 * Rows [row_begin, row_end) of the exact kNN graph of the n points x (FP32,
 * row-major n x m).  nbr / nbr_d2 hold (row_end - row_begin) x k entries.
 * Returns 0, or -1 when k is outside [1, n - 1].
 */
static void knn_row(const float* x, int64_t n, int32_t m, int32_t k, int64_t i, int32_t* bj, double* bd);

int oracle_knn(const float* x, int64_t n, int32_t m, int32_t k, int64_t row_begin, int64_t row_end,
               int32_t* nbr, double* nbr_d2)
{
    if (k < 1 || (int64_t)k > n - 1 || row_begin < 0 || row_end > n || row_begin > row_end) return -1;
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = row_begin; i < row_end; ++i)
        knn_row(x, n, m, k, i, nbr + (i - row_begin) * k, nbr_d2 + (i - row_begin) * k);
    return 0;
}

/* The same search for an explicit list of rows (rows[t] -> output row t). */
int oracle_knn_rows(const float* x, int64_t n, int32_t m, int32_t k, const int64_t* rows, int64_t nrows,
                    int32_t* nbr, double* nbr_d2)
{
    if (k < 1 || (int64_t)k > n - 1) return -1;
    for (int64_t t = 0; t < nrows; ++t)
        if (rows[t] < 0 || rows[t] >= n) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nrows; ++t)
        knn_row(x, n, m, k, rows[t], nbr + t * k, nbr_d2 + t * k);
    return 0;
}

static void knn_row(const float* x, int64_t n, int32_t m, int32_t k, int64_t i, int32_t* bj, double* bd)
{
    {
        int32_t cnt = 0;
        const float* xi = x + i * m;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d = canon_d2(xi, x + j * m, m);
            /* candidate enters when the list is short or it precedes the last kept entry */
            if (cnt == k && !(d < bd[k - 1] || (d == bd[k - 1] && j < bj[k - 1]))) continue;
            int32_t pos = (cnt < k) ? cnt++ : k - 1;
            while (pos > 0 && (d < bd[pos - 1] || (d == bd[pos - 1] && j < bj[pos - 1]))) {
                bd[pos] = bd[pos - 1];
                bj[pos] = bj[pos - 1];
                --pos;
            }
            bd[pos] = d;
            bj[pos] = (int32_t)j;
        }
    }
}
