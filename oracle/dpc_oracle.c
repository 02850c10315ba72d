/*
 * CPU oracle for exact Density-Peaks Clustering (DPC).
 *
 * TEST INFRASTRUCTURE. This is the plain, slow, obviously correct reference
 * that the CUDA library is checked against. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may build, load or run it. It
 * shares no code, header, table or helper with the CUDA library, and the
 * library never calls it.
 *
 * What it computes follows the paper's problem definition (Section 2.1,
 * Definitions 1-6) and its straightforward "Scan" algorithm (Section 2.2):
 * a linear scan for every local density, a sort by density, a scan of the
 * denser prefix for every dependent point, and a depth-first label
 * propagation from the cluster centers. OpenMP spreads the independent
 * per-point loops over the host cores; it changes no arithmetic.
 *
 * Readings of the paper (it is silent or loose on these points):
 *  - dist() is Euclidean. It is compared squared, exactly, in 64-bit
 *    integers: D(i,j) = sum_k (x_ik - x_jk)^2. Coordinates are int32 in
 *    [0, 2^30), so D < 2^63.
 *  - Definition 1 ranges over every p_j in P, so p_i counts itself; "less
 *    than d_cut" is strict: rho_i = #{ j : D(i,j) < d_cut^2 }.
 *  - "Higher density" is the total order (rho desc, index asc). This is what
 *    Ex-DPC computes (Section 3: sort by density, pop the front, search the
 *    points already inserted) when its sort is stable, and it replaces the
 *    paper's random (0,1) tie-breaker by a deterministic one.
 *  - Ties in distance (Definition 2: "broken arbitrarily") go to the
 *    smallest original index.
 *  - The top point (rank 0) has no dependent point: dep = -1 and
 *    delta2 = INT64_MAX stands for delta = infinity (Definition 3).
 *  - Noise: rho_i < rho_min (Definition 4). Center: not noise and
 *    delta_i >= delta_min, tested as delta2_i >= delta_min^2 (Definition 5).
 *  - Label: the original index of the center a point reaches through its
 *    chain of dependent points (Definition 6); -1 for noise.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Squared Euclidean distance between rows i and j of the n x d row-major
 * int32 matrix P, exact in 64-bit integers. */
static int64_t sq_dist(const int32_t* P, int32_t d, int64_t i, int64_t j) {
    int64_t s = 0;
    for (int32_t k = 0; k < d; ++k) {
        int64_t t = (int64_t)P[i * d + k] - (int64_t)P[j * d + k];
        s += t * t;
    }
    return s;
}

/* p_j is "higher" than p_i: rho_j > rho_i, or equal density and j < i. */
static int higher(const int32_t* rho, int64_t j, int64_t i) {
    return rho[j] > rho[i] || (rho[j] == rho[i] && j < i);
}

/* Definition 1 by a linear scan of P for every point (Scan, step 1). */
void oracle_rho(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, int32_t* rho) {
    const int64_t r2 = d_cut * d_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (sq_dist(P, d, i, j) < r2) ++c;
        rho[i] = c;
    }
}

/* Definition 1 for the m points listed in idx (each scanned against all n). */
void oracle_rho_subset(const int32_t* P, int64_t n, int32_t d, int64_t d_cut,
                       const int64_t* idx, int64_t m, int32_t* rho_sub) {
    const int64_t r2 = d_cut * d_cut;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < m; ++t) {
        const int64_t i = idx[t];
        int32_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (sq_dist(P, d, i, j) < r2) ++c;
        rho_sub[t] = c;
    }
}

/* Scan, step 2: a stable sort of the indices by density, descending. A
 * counting sort over the density values is stable by construction, so equal
 * densities keep ascending index order. order[r] = index of rank r. */
void oracle_rank_order(const int32_t* rho, int64_t n, int64_t* order) {
    int32_t rmax = 0;
    for (int64_t i = 0; i < n; ++i)
        if (rho[i] > rmax) rmax = rho[i];
    int64_t* start = (int64_t*)calloc((size_t)rmax + 2, sizeof(int64_t));
    /* bucket b holds density rmax - b, so bucket 0 is the densest */
    for (int64_t i = 0; i < n; ++i) start[rmax - rho[i] + 1]++;
    for (int32_t b = 0; b <= rmax; ++b) start[b + 1] += start[b];
    for (int64_t i = 0; i < n; ++i) order[start[rmax - rho[i]]++] = i;
    free(start);
}

/* Scan, step 3 (Definitions 2-3): the dependent point of the point at rank r
 * is the nearest point among ranks 0..r-1, scanned front to back; the scan
 * stops at the point itself, which is Scan's early termination. Ties in
 * distance go to the smaller original index. */
void oracle_dependent(const int32_t* P, int64_t n, int32_t d, const int32_t* rho,
                      int32_t* dep, int64_t* delta2) {
    if (n <= 0) return;
    int64_t* order = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    oracle_rank_order(rho, n, order);
    dep[order[0]] = -1;
    delta2[order[0]] = INT64_MAX;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 1; r < n; ++r) {
        const int64_t i = order[r];
        int64_t best_d = INT64_MAX, best_j = -1;
        for (int64_t t = 0; t < r; ++t) {
            const int64_t j = order[t];
            const int64_t dij = sq_dist(P, d, i, j);
            if (dij < best_d || (dij == best_d && j < best_j)) {
                best_d = dij;
                best_j = j;
            }
        }
        dep[i] = (int32_t)best_j;
        delta2[i] = best_d;
    }
    free(order);
}

/* Definitions 2-3 for the m points listed in idx, straight from the
 * definition: every j in P that is higher than i is a candidate. */
void oracle_dependent_subset(const int32_t* P, int64_t n, int32_t d, const int32_t* rho,
                             const int64_t* idx, int64_t m, int32_t* dep_sub,
                             int64_t* delta2_sub) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < m; ++t) {
        const int64_t i = idx[t];
        int64_t best_d = INT64_MAX, best_j = -1;
        for (int64_t j = 0; j < n; ++j) {
            if (!higher(rho, j, i)) continue;
            const int64_t dij = sq_dist(P, d, i, j);
            if (dij < best_d || (dij == best_d && j < best_j)) {
                best_d = dij;
                best_j = j;
            }
        }
        dep_sub[t] = (int32_t)best_j;
        delta2_sub[t] = best_d;
    }
}

/* Scan, step 4 (Definitions 4-6): mark noise and centers, then propagate each
 * center's label depth-first along the reversed dependent links (every point
 * keeps the list of points that depend on it). Returns the number of centers.
 * delta_min is an integer > d_cut and delta_min^2 must fit in int64. */
int64_t oracle_label(int64_t n, const int32_t* rho, const int32_t* dep, const int64_t* delta2,
                     int64_t rho_min, int64_t delta_min, int32_t* label) {
    const int64_t dmin2 = delta_min * delta_min;
    /* children lists in CSR form: child_start[p] .. child_start[p+1] */
    int64_t* child_start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* child = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* stack = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        if (dep[i] >= 0) child_start[dep[i] + 1]++;
    for (int64_t p = 0; p < n; ++p) child_start[p + 1] += child_start[p];
    {
        int64_t* fill = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        for (int64_t p = 0; p < n; ++p) fill[p] = child_start[p];
        for (int64_t i = 0; i < n; ++i)
            if (dep[i] >= 0) child[fill[dep[i]]++] = i;
        free(fill);
    }
    for (int64_t i = 0; i < n; ++i) label[i] = -1;
    int64_t n_centers = 0;
    for (int64_t c = 0; c < n; ++c) {
        const int noise = (int64_t)rho[c] < rho_min;
        const int center = !noise && delta2[c] >= dmin2;
        if (!center) continue;
        ++n_centers;
        /* depth-first search from the center; it does not cross into other
         * centers (they start their own cluster) or into noise */
        int64_t top = 0;
        stack[top++] = c;
        label[c] = (int32_t)c;
        while (top > 0) {
            const int64_t p = stack[--top];
            for (int64_t e = child_start[p]; e < child_start[p + 1]; ++e) {
                const int64_t q = child[e];
                if ((int64_t)rho[q] < rho_min) continue;
                if (delta2[q] >= dmin2) continue;
                label[q] = (int32_t)c;
                stack[top++] = q;
            }
        }
    }
    free(child_start);
    free(child);
    free(stack);
    return n_centers;
}
