/*
 * Streaming Gram update on the host cores: the streaming method of snapshots
 * run on a CPU (Sec. 3.1, Eq. 12a-b; the update step of Algorithm 1), the
 * paper's "streaming CPU" configuration. Benchmark and test infrastructure,
 * like the rest of oracle/: bench.py times it beside the GPU path; nothing in
 * the product package calls it.
 *
 * The window lives in a ring of m slots, slot s at ring + s * pitch; the
 * slots in use are 0 .. used - 1 (the ring fills from slot 0, then the oldest
 * slot is overwritten). A push
 *   1. copies the new snapshot into slot s_new,
 *   2. computes its inner product with every slot in use (itself included),
 *        g_j = <x_j, x_new>,   j = 0 .. used - 1,
 *   3. writes g as row and column s_new of the physical Gram G (m x m,
 *      row-major). No other entry of G moves: the oldest row and column are
 *      overwritten in place.
 *
 * 8-bit snapshots: exact int64. The positions are cut into blocks of 32768;
 * a block's sum of products fits in uint32 (32768 * 255^2 < 2^32) and is then
 * added in int64. Blocks are spread over the host threads when OpenMP is
 * available; each thread keeps its own partial g, added at the end, so the
 * integer result does not depend on the split.
 *
 * FP32 snapshots: products and sums in FP64; a thread's partial sums follow
 * the position order within its blocks, and the partials of the threads are
 * added in an order that depends on the thread count, so results agree with
 * one sequential FP64 sum to rounding.
 */
#include <stdint.h>
#include <string.h>

#define SCPU_BLOCK 32768
#define SCPU_MAX_M 256

int scpu_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int scpu_push_u8(uint8_t *ring, int64_t pitch, int64_t n, int32_t m, int32_t used, int32_t s_new,
                 const uint8_t *x, int64_t *G) {
    if (m < 1 || m > SCPU_MAX_M || used < 1 || used > m || s_new < 0 || s_new >= used || n < 0 ||
        pitch < n)
        return -1;
    uint8_t *dst = ring + (int64_t)s_new * pitch;
    const int64_t nb = (n + SCPU_BLOCK - 1) / SCPU_BLOCK;
    int64_t g[SCPU_MAX_M];
    for (int32_t j = 0; j < used; ++j) g[j] = 0;
#pragma omp parallel
    {
        int64_t part[SCPU_MAX_M];
        for (int32_t j = 0; j < used; ++j) part[j] = 0;
#pragma omp for schedule(static)
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t k0 = b * SCPU_BLOCK;
            const int64_t len = (n - k0 < SCPU_BLOCK) ? n - k0 : SCPU_BLOCK;
            memcpy(dst + k0, x + k0, (size_t)len);
            const uint8_t *xn = x + k0;
            for (int32_t j = 0; j < used; ++j) {
                const uint8_t *xj = ring + (int64_t)j * pitch + k0;
                uint32_t s = 0;
                for (int64_t k = 0; k < len; ++k) s += (uint32_t)xj[k] * (uint32_t)xn[k];
                part[j] += (int64_t)s;
            }
        }
#pragma omp critical
        for (int32_t j = 0; j < used; ++j) g[j] += part[j];
    }
    for (int32_t j = 0; j < used; ++j) {
        G[(int64_t)s_new * m + j] = g[j];
        G[(int64_t)j * m + s_new] = g[j];
    }
    return 0;
}

/* pitch in elements (floats) */
int scpu_push_f32(float *ring, int64_t pitch, int64_t n, int32_t m, int32_t used, int32_t s_new,
                  const float *x, double *G) {
    if (m < 1 || m > SCPU_MAX_M || used < 1 || used > m || s_new < 0 || s_new >= used || n < 0 ||
        pitch < n)
        return -1;
    float *dst = ring + (int64_t)s_new * pitch;
    const int64_t nb = (n + SCPU_BLOCK - 1) / SCPU_BLOCK;
    double g[SCPU_MAX_M];
    for (int32_t j = 0; j < used; ++j) g[j] = 0.0;
#pragma omp parallel
    {
        double part[SCPU_MAX_M];
        for (int32_t j = 0; j < used; ++j) part[j] = 0.0;
#pragma omp for schedule(static)
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t k0 = b * SCPU_BLOCK;
            const int64_t len = (n - k0 < SCPU_BLOCK) ? n - k0 : SCPU_BLOCK;
            memcpy(dst + k0, x + k0, (size_t)len * sizeof(float));
            const float *xn = x + k0;
            for (int32_t j = 0; j < used; ++j) {
                const float *xj = ring + (int64_t)j * pitch + k0;
                double s = 0.0;
                for (int64_t k = 0; k < len; ++k) s += (double)xj[k] * (double)xn[k];
                part[j] += s;
            }
        }
#pragma omp critical
        for (int32_t j = 0; j < used; ++j) g[j] += part[j];
    }
    for (int32_t j = 0; j < used; ++j) {
        G[(int64_t)s_new * m + j] = g[j];
        G[(int64_t)j * m + s_new] = g[j];
    }
    return 0;
}
