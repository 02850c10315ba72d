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
 * per-point loops over the host cores; it changes no arithmetic. The last
 * oracle_approx_* functions follow Approx-DPC's dependent-point rules
 * (Section 4.3) on top of the same exact densities; the oracle_sapprox_*
 * functions follow S-Approx-DPC (Section 5).
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
#include <math.h>
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

/* ----------------------------------------------------------------------
 * Approx-DPC's dependent points (Section 4.3, "Approximate computation"
 * and "Exact computation"), on top of exact local densities.
 *
 * The grid G has non-empty cells of side d_cut / sqrt(d) (Section 4.1).
 * Readings (the paper is silent or loose on these):
 *  - The side is the integer s = max(1, floor(d_cut / sqrt(d))), anchored
 *    at the per-dimension minimum of P: the cell of p has coordinates
 *    floor((x_k - min_k) / s). Two points of one cell are then strictly
 *    closer than d_cut, which is what the approximation rules rely on.
 *  - p*(c) is the highest point of c in the total order (rho desc, index
 *    asc) used everywhere else.
 *  - "min over P(c') of rho > rho_i" reads, in that total order, as: every
 *    point of c' is higher than p_i.
 *  - N(c) is the set of cells other than c that hold a point p with
 *    D(p*(c), p) < d_cut^2 (strict, as in Definition 1).
 *  - When several cells of N(c) qualify, the one whose p* is highest wins.
 *  - An approximated dependent distance is d_cut, i.e. delta2 = d_cut^2.
 *  - A point left undecided gets its exact dependent point (Definitions 2-3,
 *    ties to the smaller index); the top point keeps dep -1 and
 *    delta2 = INT64_MAX.
 * exact[i] is 1 when point i's dependent point is the exact one.
 */

/* floor(sqrt(a)) for 0 <= a < 2^62 (the library square root as a first
 * guess, corrected in integers). */
static int64_t isqrt_i64(int64_t a) {
    int64_t r = (int64_t)sqrt((double)a);
    while (r > 0 && r * r > a) --r;
    while ((r + 1) * (r + 1) <= a) ++r;
    return r;
}

int64_t oracle_approx_side(int64_t d_cut, int32_t d) {
    int64_t s = isqrt_i64((d_cut * d_cut) / d);
    return s < 1 ? 1 : s;
}

/* Cell coordinates of every point (n x d, int64). */
static int64_t* approx_cells(const int32_t* P, int64_t n, int32_t d, int64_t s) {
    int64_t* cc = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * d * sizeof(int64_t));
    for (int32_t k = 0; k < d; ++k) {
        int64_t lo = 0;
        for (int64_t i = 0; i < n; ++i)
            if (i == 0 || P[i * d + k] < lo) lo = P[i * d + k];
        for (int64_t i = 0; i < n; ++i) cc[i * d + k] = ((int64_t)P[i * d + k] - lo) / s;
    }
    return cc;
}

static const int64_t* g_cc;  /* qsort context: cell coordinates */
static int32_t g_d;
static int cmp_cells(const void* a, const void* b) {
    const int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
    for (int32_t k = 0; k < g_d; ++k) {
        const int64_t x = g_cc[i * g_d + k], y = g_cc[j * g_d + k];
        if (x != y) return x < y ? -1 : 1;
    }
    return i < j ? -1 : (i > j ? 1 : 0);
}

/* Dependent points of the m points listed in idx (all n when idx is NULL). */
static void approx_dependent(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, const int32_t* rho,
                             const int64_t* idx, int64_t m, int32_t* dep_out, int64_t* delta2_out,
                             int32_t* exact_out) {
    if (n <= 0) return;
    const int64_t r2 = d_cut * d_cut;
    const int64_t s = oracle_approx_side(d_cut, d);
    int64_t* cc = approx_cells(P, n, d, s);
    /* rank of every point */
    int64_t* order = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* rank = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    oracle_rank_order(rho, n, order);
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = r;
    /* group the points by cell: sort by cell coordinates, then number the cells */
    int64_t* by_cell = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) by_cell[i] = i;
    g_cc = cc;
    g_d = d;
    qsort(by_cell, (size_t)n, sizeof(int64_t), cmp_cells);
    int64_t* cell = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* pstar = (int64_t*)malloc((size_t)n * sizeof(int64_t));    /* per cell: highest point */
    int64_t* maxrank = (int64_t*)malloc((size_t)n * sizeof(int64_t));  /* per cell: lowest point's rank */
    int64_t ncell = 0;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t i = by_cell[t];
        int same = 0;
        if (t > 0) {
            const int64_t j = by_cell[t - 1];
            same = 1;
            for (int32_t k = 0; k < d; ++k)
                if (cc[i * d + k] != cc[j * d + k]) same = 0;
        }
        if (!same) {
            pstar[ncell] = i;
            maxrank[ncell] = rank[i];
            ++ncell;
        }
        const int64_t c = ncell - 1;
        cell[i] = c;
        if (rank[i] < rank[pstar[c]]) pstar[c] = i;
        if (rank[i] > maxrank[c]) maxrank[c] = rank[i];
    }
    const int64_t count = idx ? m : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < count; ++t) {
        const int64_t i = idx ? idx[t] : t;
        const int64_t c = cell[i];
        int64_t dp = -1, d2 = INT64_MAX;
        int32_t ex = 0;
        if (pstar[c] != i) {
            /* rule 1: the highest point of the own cell */
            dp = pstar[c];
            d2 = r2;
        } else {
            /* rule 2: a cell of N(c) whose points are all higher than p_i */
            int64_t best = -1;
            for (int64_t j = 0; j < n; ++j) {
                const int64_t cj = cell[j];
                if (cj == c || sq_dist(P, d, i, j) >= r2) continue;
                if (maxrank[cj] < rank[i] && (best < 0 || rank[pstar[cj]] < rank[best])) best = pstar[cj];
            }
            if (best >= 0) {
                dp = best;
                d2 = r2;
            } else {
                /* exact computation: the nearest higher point */
                ex = 1;
                for (int64_t j = 0; j < n; ++j) {
                    if (rank[j] >= rank[i]) continue;
                    const int64_t dij = sq_dist(P, d, i, j);
                    if (dij < d2 || (dij == d2 && j < dp)) {
                        d2 = dij;
                        dp = j;
                    }
                }
            }
        }
        dep_out[t] = (int32_t)dp;
        delta2_out[t] = d2;
        if (exact_out) exact_out[t] = ex;
    }
    free(cc);
    free(order);
    free(rank);
    free(by_cell);
    free(cell);
    free(pstar);
    free(maxrank);
}

void oracle_approx_dependent(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, const int32_t* rho,
                             int32_t* dep, int64_t* delta2, int32_t* exact) {
    approx_dependent(P, n, d, d_cut, rho, NULL, n, dep, delta2, exact);
}

void oracle_approx_dependent_subset(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, const int32_t* rho,
                                    const int64_t* idx, int64_t m, int32_t* dep_sub, int64_t* delta2_sub,
                                    int32_t* exact_sub) {
    approx_dependent(P, n, d, d_cut, rho, idx, m, dep_sub, delta2_sub, exact_sub);
}

/* ----------------------------------------------------------------------
 * S-Approx-DPC (Section 5): one picked point per cell of the grid G' of
 * side eps * d_cut / sqrt(d); local densities and dependent points of the
 * picked points only; every other point depends on its cell's pick.
 *
 * Readings (the paper leaves these choices open or loose):
 *  - eps = eps_num / eps_den; the side is the integer
 *    s = max(1, floor(eps * d_cut / sqrt(d))), anchored at the
 *    per-dimension minimum of P.
 *  - The picked point of a cell ("decided in an arbitrary way") is its point
 *    with the smallest original index.
 *  - A pick's local density is Definition 1 against all of P. Picks are
 *    ordered by (rho desc, index asc); "higher" compares picks only.
 *  - N(c): the cells other than c holding a point p' with
 *    D(pick(c), p') < d_cut^2.
 *  - First phase: among the picks of the cells in N(c) that are higher than
 *    pick(c) (chosen "arbitrarily" in the paper), the nearest one, ties to
 *    the smaller index; its exact squared distance is the delta2.
 *  - Second phase: a pick without such a candidate gets its nearest higher
 *    pick over all picks (what the paper's temporary-cluster pruning finds
 *    exactly); the highest pick keeps dep -1 and delta2 INT64_MAX.
 *  - A point that is not picked: dep = its cell's pick, delta2 = its exact
 *    squared distance to it, rho = -1 (not computed).
 * pick[i] is 1 for the picked points.
 */
int64_t oracle_sapprox_side(int64_t d_cut, int32_t d, int64_t eps_num, int64_t eps_den) {
    /* floor(eps * d_cut / sqrt(d)) = floor(sqrt((eps_num d_cut)^2 / (eps_den^2 d))) */
    const double num = (double)eps_num * (double)d_cut;
    const int64_t q = (int64_t)((num * num) / ((double)eps_den * (double)eps_den * (double)d));
    int64_t s = isqrt_i64(q);
    /* q may be off by rounding of the double quotient: correct s exactly */
    while (s > 0 && (__int128)s * s * eps_den * eps_den * d > (__int128)eps_num * eps_num * d_cut * d_cut) --s;
    while ((__int128)(s + 1) * (s + 1) * eps_den * eps_den * d <= (__int128)eps_num * eps_num * d_cut * d_cut) ++s;
    return s < 1 ? 1 : s;
}

/* The grid G' and its picks: cell[i] is the index of point i's cell (cells
 * numbered in sorted cell order), cpick[c] the pick of cell c, pick[i] 1 for
 * the picks. */
static void sapprox_grid(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, int64_t eps_num, int64_t eps_den,
                         int64_t* cell, int64_t* cpick, int32_t* pick) {
    const int64_t s = oracle_sapprox_side(d_cut, d, eps_num, eps_den);
    int64_t* cc = approx_cells(P, n, d, s);
    int64_t* by_cell = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) by_cell[i] = i;
    g_cc = cc;
    g_d = d;
    qsort(by_cell, (size_t)n, sizeof(int64_t), cmp_cells);
    int64_t ncell = 0;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t i = by_cell[t];
        int same = 0;
        if (t > 0) {
            const int64_t j = by_cell[t - 1];
            same = 1;
            for (int32_t k = 0; k < d; ++k)
                if (cc[i * d + k] != cc[j * d + k]) same = 0;
        }
        if (!same) cpick[ncell++] = i;
        const int64_t c = ncell - 1;
        cell[i] = c;
        if (i < cpick[c]) cpick[c] = i;
    }
    for (int64_t i = 0; i < n; ++i) pick[i] = cpick[cell[i]] == i;
    free(cc);
    free(by_cell);
}

/* The dependent point of point i (rho given for every pick). */
static void sapprox_link(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, const int64_t* cell,
                         const int64_t* cpick, const int32_t* pick, const int32_t* rho, int64_t i, int32_t* dep_i,
                         int64_t* delta2_i) {
    const int64_t r2 = d_cut * d_cut;
    if (!pick[i]) {
        *dep_i = (int32_t)cpick[cell[i]];
        *delta2_i = sq_dist(P, d, i, cpick[cell[i]]);
        return;
    }
    /* pick q is higher than pick i: rho_q > rho_i, or equal and q < i */
    int64_t dp = -1, d2 = INT64_MAX;
    /* first phase: picks of the cells of N(c) */
    for (int64_t j = 0; j < n; ++j) {
        if (cell[j] == cell[i] || sq_dist(P, d, i, j) >= r2) continue;
        const int64_t q = cpick[cell[j]];
        if (!(rho[q] > rho[i] || (rho[q] == rho[i] && q < i))) continue;
        const int64_t dq = sq_dist(P, d, i, q);
        if (dq < d2 || (dq == d2 && q < dp)) {
            d2 = dq;
            dp = q;
        }
    }
    if (dp < 0) {
        /* second phase: the nearest higher pick over all picks */
        for (int64_t q = 0; q < n; ++q) {
            if (!pick[q] || !(rho[q] > rho[i] || (rho[q] == rho[i] && q < i))) continue;
            const int64_t dq = sq_dist(P, d, i, q);
            if (dq < d2 || (dq == d2 && q < dp)) {
                d2 = dq;
                dp = q;
            }
        }
    }
    *dep_i = (int32_t)dp;
    *delta2_i = d2;
}

void oracle_sapprox(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, int64_t eps_num, int64_t eps_den,
                    int32_t* rho, int32_t* dep, int64_t* delta2, int32_t* pick) {
    if (n <= 0) return;
    const int64_t r2 = d_cut * d_cut;
    int64_t* cell = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* cpick = (int64_t*)malloc((size_t)n * sizeof(int64_t));  /* per cell: its pick */
    sapprox_grid(P, n, d, d_cut, eps_num, eps_den, cell, cpick, pick);
    /* densities of the picks (Definition 1 against all points) */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        if (!pick[i]) {
            rho[i] = -1;
            continue;
        }
        int32_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (sq_dist(P, d, i, j) < r2) ++c;
        rho[i] = c;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) sapprox_link(P, n, d, d_cut, cell, cpick, pick, rho, i, &dep[i], &delta2[i]);
    free(cell);
    free(cpick);
}

/* The sampled form for sets too large for the full one: picks and links of
 * the points idx[0..m), given rho for every pick (the other entries are not
 * read). The picks' densities themselves are checked with oracle_rho_subset. */
void oracle_sapprox_dependent_subset(const int32_t* P, int64_t n, int32_t d, int64_t d_cut, int64_t eps_num,
                                     int64_t eps_den, const int32_t* rho, const int64_t* idx, int64_t m,
                                     int32_t* dep_sub, int64_t* delta2_sub, int32_t* pick_sub) {
    if (n <= 0) return;
    int64_t* cell = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* cpick = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int32_t* pick = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    sapprox_grid(P, n, d, d_cut, eps_num, eps_den, cell, cpick, pick);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < m; ++t) {
        sapprox_link(P, n, d, d_cut, cell, cpick, pick, rho, idx[t], &dep_sub[t], &delta2_sub[t]);
        pick_sub[t] = pick[idx[t]];
    }
    free(cell);
    free(cpick);
    free(pick);
}

/* Labels of S-Approx-DPC: Definitions 4-6 over the picks (noise: rho below
 * rho_min; centers: non-noise picks with delta2 >= delta_min^2; labels along
 * the dependent links among picks), then every other point takes its pick's
 * label (rho_min does not apply to it). Returns the number of centers. */
int64_t oracle_sapprox_label(int64_t n, const int32_t* rho, const int32_t* dep, const int64_t* delta2,
                             const int32_t* pick, int64_t rho_min, int64_t delta_min, int32_t* label) {
    const int64_t dmin2 = delta_min * delta_min;
    int64_t n_centers = 0;
    for (int64_t i = 0; i < n; ++i) label[i] = -2; /* not yet known */
    for (int64_t i = 0; i < n; ++i) {
        if (!pick[i]) continue;
        if ((int64_t)rho[i] < rho_min) label[i] = -1;
        else if (delta2[i] >= dmin2) {
            label[i] = (int32_t)i;
            ++n_centers;
        }
    }
    /* follow each pick's chain to the first labelled pick (a center, or the
     * densest pick, which is a center unless it is noise) */
    for (int64_t i = 0; i < n; ++i) {
        if (!pick[i] || label[i] != -2) continue;
        int64_t q = i, hops = 0;
        while (label[q] == -2 && dep[q] >= 0 && hops <= n) {
            q = dep[q];
            ++hops;
        }
        const int32_t l = label[q] == -2 ? -1 : label[q];
        /* write the label along the chain */
        int64_t r = i;
        while (label[r] == -2) {
            label[r] = l;
            if (dep[r] < 0) break;
            r = dep[r];
        }
    }
    for (int64_t i = 0; i < n; ++i)
        if (!pick[i]) label[i] = label[dep[i]];
    return n_centers;
}
