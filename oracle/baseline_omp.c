/*
 * baseline_omp.c - timing context only, not a parity reference.
 *
 * The oracle's Jacobi sweep (Eq. 1: every interior vertex moves to the mean of
 * its neighbours' positions, each coordinate summed left to right over the
 * stored row from 0.0 and divided once by the neighbour count; boundary
 * vertices keep their place) with the vertex loop shared between host threads
 * by an OpenMP static schedule, as the paper's Section 5.1 runs its sweeps on
 * 32 cores.  Used only by the benchmark's CPU-baseline leg to time the method on
 * every host core.  Each vertex's arithmetic is the oracle's, so the result
 * equals the single-thread oracle bit for bit at any thread count (checked by a
 * CPU test).  Test infrastructure: the library never links or calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* iters simultaneous sweeps of xy ([2n], in place; one scratch buffer); threads <= 0: OpenMP's default.
   Returns the thread count used, or -1 on a bad argument / allocation failure. */
int bl_jacobi_omp(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                  double* xy, int32_t iters, int32_t threads) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !xy || iters < 0) return -1;
    double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!tmp) return -1;
    if (threads > 0) omp_set_num_threads(threads);
    int used = 1;
    double* src = xy;
    double* dst = tmp;
    for (int32_t k = 0; k < iters; ++k) {
#pragma omp parallel
        {
#pragma omp single
            used = omp_get_num_threads();
#pragma omp for schedule(static)
            for (int32_t v = 0; v < n; ++v) {
                if (is_boundary[v]) {
                    dst[2 * v] = src[2 * v];
                    dst[2 * v + 1] = src[2 * v + 1];
                    continue;
                }
                double sx = 0.0, sy = 0.0;
                const int32_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t u = col_idx[e];
                    sx = sx + src[2 * u];
                    sy = sy + src[2 * u + 1];
                }
                dst[2 * v] = sx / (double)(e1 - e0);
                dst[2 * v + 1] = sy / (double)(e1 - e0);
            }
        }
        double* t = src;
        src = dst;
        dst = t;
    }
    if (src != xy) memcpy(xy, src, sizeof(double) * 2 * (size_t)n);
    free(tmp);
    return used;
}
