/*
 * Direct FP64 Cauchy sum on the host cores (OpenMP).
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle, used by the tests and by
 * the benchmark's CPU baseline; the CUDA library never links or calls it.
 *
 * Computes the Cauchy sum of Sec. 2.5, Eq. (fmm-E), straight from its
 * definition:
 *     z_i = sum_{j != i} w_j / (eta_i - eta_j),   i = 0 .. N-1,
 * each term as w_j conj(d) / |d|^2 with d = eta_i - eta_j, one row per loop
 * iteration (rows split over `threads` OpenMP threads, each row summed in
 * order j = 0 .. N-1, so the result does not depend on the thread count).
 * et, w, z: interleaved (re, im) doubles, 2N each.
 */
#include <omp.h>

void oracle_cauchy_sum(int N, const double* et, const double* w, double* z, int threads) {
    if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) {
        const double xr = et[2 * i], xi = et[2 * i + 1];
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            const double dr = xr - et[2 * j], di = xi - et[2 * j + 1];
            const double inv = 1.0 / (dr * dr + di * di);
            const double wr = w[2 * j], wi = w[2 * j + 1];
            sr += (wr * dr + wi * di) * inv;
            si += (wi * dr - wr * di) * inv;
        }
        z[2 * i] = sr;
        z[2 * i + 1] = si;
    }
}
