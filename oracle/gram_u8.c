/*
 * Oracle (test infrastructure only): exact Gram matrix of 8-bit snapshots.
 *
 * The method of snapshots needs the inner-product matrix X*X of the window
 * (Sec. 2.1, Eq. 3; streaming form Sec. 3.1, Eq. 12a-b). For 8-bit pixels the
 * plain definition G[i][j] = sum_k x_i[k] * x_j[k] is an integer, accumulated
 * here in int64 with no blocking or reordering: one product, one add.
 *
 * cols[i] points at snapshot i (n bytes). G is c x c, row-major, int64.
 * The pair loop runs across host threads when OpenMP is available; each
 * entry is still one sequential exact sum, so the result is unique.
 */
#include <stdint.h>

int64_t oracle_dot_u8(const uint8_t *a, const uint8_t *b, int64_t n) {
    int64_t s = 0;
    for (int64_t k = 0; k < n; ++k) s += (int64_t)a[k] * (int64_t)b[k];
    return s;
}

void oracle_gram_u8(const uint8_t *const *cols, int64_t n, int32_t c, int64_t *G) {
    int64_t npairs = (int64_t)c * (c + 1) / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < npairs; ++q) {
        /* q -> (i, j) with i <= j, row by row of the upper triangle */
        int32_t i = 0;
        int64_t rem = q;
        while (rem >= c - i) { rem -= c - i; ++i; }
        int32_t j = i + (int32_t)rem;
        int64_t s = oracle_dot_u8(cols[i], cols[j], n);
        G[(int64_t)i * c + j] = s;
        G[(int64_t)j * c + i] = s;
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
