/*
 * Oracle for exact k-nearest neighbours and friends-of-friends (FoF) groups.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA path.
 *
 * Definitions followed (all arithmetic in float64 on the float32 inputs):
 *   kNN  (Sec. III, problem statement): for each query i, the k points j
 *        (i itself included) with the smallest squared distance d2(i,j),
 *        ties broken by the lower index j.
 *   FoF  (Sec. IV, eq. for R_link and the linking rule of Sec. IV-A): connected
 *        components of the graph with an edge between i and j when
 *        d2(i,j) <= b2; every point is labelled with the smallest index in
 *        its component.
 *   Periodic boxes (Sec. III-G, "periodic wrapping"): L > 0 means coordinates
 *        live in [0,L)^3 and each coordinate difference is replaced by its
 *        minimum image  d - L*round(d/L).
 *
 * Two implementations of each: an all-pairs one (obviously correct, O(N^2))
 * and a cell-list one (exact, for large N) that the tests check against the
 * all-pairs one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ basics */

static double pair_d2(const float *a, const float *b, double L)
{
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        double d = (double)b[c] - (double)a[c];
        if (L > 0.0)
            d -= L * round(d / L);
        d2 += d * d;
    }
    return d2;
}

/* insert (d, j) into the ascending list (kd, ki) of current length *m <= k,
 * ordered by (d, j); returns nothing, keeps at most k entries. */
static void topk_insert(double *kd, int32_t *ki, int *m, int k, double d, int32_t j)
{
    int n = *m;
    if (n == k) {
        double wd = kd[k - 1];
        int32_t wi = ki[k - 1];
        if (d > wd || (d == wd && j >= wi))
            return;
        n = k - 1; /* drop the current worst */
    }
    int pos = n;
    while (pos > 0 && (kd[pos - 1] > d || (kd[pos - 1] == d && ki[pos - 1] > j))) {
        kd[pos] = kd[pos - 1];
        ki[pos] = ki[pos - 1];
        --pos;
    }
    kd[pos] = d;
    ki[pos] = j;
    *m = n + 1;
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_num_threads(int nthreads) { return set_threads(nthreads); }

/* ------------------------------------------------------------- all-pairs kNN
 * queries: nq indices into xyz (or NULL for all N points, nq == n).
 * out_idx / out_d2: nq x k, row r is ascending by (d2, j). */
int oracle_knn_brute(const float *xyz, int64_t n, int k, double L,
                     const int64_t *queries, int64_t nq,
                     int32_t *out_idx, double *out_d2, int nthreads)
{
    if (n < 1 || k < 1 || k > n)
        return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nq; ++r) {
        int64_t i = queries ? queries[r] : r;
        double *kd = out_d2 + r * k;
        int32_t *ki = out_idx + r * k;
        int m = 0;
        for (int64_t j = 0; j < n; ++j)
            topk_insert(kd, ki, &m, k, pair_d2(xyz + 3 * i, xyz + 3 * j, L), (int32_t)j);
    }
    return 0;
}

/* ---------------------------------------------------------------- union-find
 * Linking always points the larger root at the smaller one, so the root of
 * every set is its smallest member. */
static int64_t uf_find(int64_t *p, int64_t x)
{
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

static void uf_union(int64_t *p, int64_t a, int64_t b)
{
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b)
        return;
    if (a < b)
        p[b] = a;
    else
        p[a] = b;
}

/* ------------------------------------------------------------- all-pairs FoF */
int oracle_fof_brute(const float *xyz, int64_t n, double b2, double L, int32_t *labels)
{
    if (n < 1)
        return -1;
    int64_t *p = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!p)
        return -2;
    for (int64_t i = 0; i < n; ++i)
        p[i] = i;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (pair_d2(xyz + 3 * i, xyz + 3 * j, L) <= b2)
                uf_union(p, i, j);
    for (int64_t i = 0; i < n; ++i)
        labels[i] = (int32_t)uf_find(p, i);
    free(p);
    return 0;
}

/* ------------------------------------------------------------ grid helpers */
typedef struct {
    double lo[3];   /* grid origin */
    double w[3];    /* cell width per dimension */
    int64_t g[3];   /* cells per dimension */
    double L;       /* > 0: periodic box side */
} grid_t;

static void grid_box(const float *xyz, int64_t n, double L, double lo[3], double hi[3])
{
    if (L > 0.0) {
        for (int c = 0; c < 3; ++c) {
            lo[c] = 0.0;
            hi[c] = L;
        }
        return;
    }
    for (int c = 0; c < 3; ++c) {
        lo[c] = INFINITY;
        hi[c] = -INFINITY;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            double v = xyz[3 * i + c];
            if (v < lo[c]) lo[c] = v;
            if (v > hi[c]) hi[c] = v;
        }
}

static int64_t cell_coord(const grid_t *g, double v, int c)
{
    double t = floor((v - g->lo[c]) / g->w[c]);
    if (t < 0.0) t = 0.0;
    if (t > (double)(g->g[c] - 1)) t = (double)(g->g[c] - 1);
    return (int64_t)t;
}

/* --------------------------------------------------------- cell-list kNN
 * Dense grid of about n/2 cells; points bucketed by cell with a counting sort
 * (stable, so indices ascend within a cell).  A query visits Chebyshev shells
 * s = 0,1,2,... of cells around its own cell and stops once every unvisited
 * point is provably farther than the current k-th distance: such a point lies
 * outside the (2s+1)^3 block of visited cells in some dimension, so its
 * distance is at least the query's distance to the nearest block face.  The
 * stop test is strict (lb^2 > d2_k), so points tied with the k-th distance are
 * still visited and the index tie-break stays exact.  In a periodic box the
 * search falls back to all pairs once the block would wrap onto itself. */
int oracle_knn_cells(const float *xyz, int64_t n, int k, double L,
                     const int64_t *queries, int64_t nq,
                     int32_t *out_idx, double *out_d2, int nthreads)
{
    if (n < 1 || k < 1 || k > n)
        return -1;
    set_threads(nthreads);
    double lo[3], hi[3];
    grid_box(xyz, n, L, lo, hi);
    double side = 0.0;
    for (int c = 0; c < 3; ++c)
        side = fmax(side, hi[c] - lo[c]);
    if (!(side > 0.0))
        side = 1.0;
    int64_t gs = (int64_t)floor(cbrt((double)n / 2.0));
    if (gs < 1) gs = 1;
    if (gs > 512) gs = 512;
    grid_t g;
    g.L = L;
    for (int c = 0; c < 3; ++c) {
        g.lo[c] = lo[c];
        g.g[c] = gs;
        /* open: widen by a hair so the maximum lands inside the last cell */
        g.w[c] = (L > 0.0) ? L / (double)gs : side * (1.0 + 1e-12) / (double)gs;
    }
    int64_t ncell = gs * gs * gs;
    int32_t *start = (int32_t *)calloc((size_t)ncell + 1, sizeof(int32_t));
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *cid = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!start || !order || !cid) {
        free(start); free(order); free(cid);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = cell_coord(&g, xyz[3 * i + 0], 0);
        int64_t cy = cell_coord(&g, xyz[3 * i + 1], 1);
        int64_t cz = cell_coord(&g, xyz[3 * i + 2], 2);
        cid[i] = (cx * gs + cy) * gs + cz;
        start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c)
        start[c + 1] += start[c];
    {
        int32_t *fill = (int32_t *)malloc((size_t)ncell * sizeof(int32_t));
        if (!fill) {
            free(start); free(order); free(cid);
            return -2;
        }
        memcpy(fill, start, (size_t)ncell * sizeof(int32_t));
        for (int64_t i = 0; i < n; ++i)
            order[fill[cid[i]]++] = (int32_t)i;
        free(fill);
    }
    const double eps = 1e-9 * side;

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nq; ++r) {
        int64_t i = queries ? queries[r] : r;
        const float *q = xyz + 3 * i;
        double *kd = out_d2 + r * k;
        int32_t *ki = out_idx + r * k;
        int m = 0;
        int64_t cc[3];
        for (int c = 0; c < 3; ++c)
            cc[c] = cell_coord(&g, q[c], c);
        int brute = 0;
        for (int64_t s = 0;; ++s) {
            if (L > 0.0 && 2 * s + 1 > gs) {
                brute = 1;
                break;
            }
            /* visit the cells of shell s */
            for (int64_t dx = -s; dx <= s; ++dx)
                for (int64_t dy = -s; dy <= s; ++dy)
                    for (int64_t dz = -s; dz <= s; ++dz) {
                        int64_t a = llabs(dx), b = llabs(dy), e = llabs(dz);
                        int64_t cheb = a > b ? a : b;
                        cheb = cheb > e ? cheb : e;
                        if (cheb != s)
                            continue;
                        int64_t c3[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
                        int ok = 1;
                        for (int c = 0; c < 3; ++c) {
                            if (L > 0.0)
                                c3[c] = ((c3[c] % gs) + gs) % gs;
                            else if (c3[c] < 0 || c3[c] >= gs)
                                ok = 0;
                        }
                        if (!ok)
                            continue;
                        int64_t cell = (c3[0] * gs + c3[1]) * gs + c3[2];
                        for (int32_t t = start[cell]; t < start[cell + 1]; ++t) {
                            int32_t j = order[t];
                            topk_insert(kd, ki, &m, k, pair_d2(q, xyz + 3 * (int64_t)j, L), j);
                        }
                    }
            /* lower bound on the distance of any point outside the block */
            double lb = INFINITY;
            int all_covered = 1;
            for (int c = 0; c < 3; ++c) {
                double blo = g.lo[c] + (double)(cc[c] - s) * g.w[c];
                double bhi = g.lo[c] + (double)(cc[c] + s + 1) * g.w[c];
                if (L > 0.0 || cc[c] - s > 0) {
                    lb = fmin(lb, (double)q[c] - blo);
                    all_covered = 0;
                }
                if (L > 0.0 || cc[c] + s < gs - 1) {
                    lb = fmin(lb, bhi - (double)q[c]);
                    all_covered = 0;
                }
            }
            if (all_covered)
                break;
            lb -= eps;
            if (m == k && lb > 0.0 && lb * lb > kd[k - 1])
                break;
        }
        if (brute) {
            m = 0;
            for (int64_t j = 0; j < n; ++j)
                topk_insert(kd, ki, &m, k, pair_d2(q, xyz + 3 * j, L), (int32_t)j);
        }
    }
    free(start);
    free(order);
    free(cid);
    return 0;
}

/* --------------------------------------------------------- cell-list FoF
 * Cells of side w <= b/sqrt(3)*(1-1e-9): the diagonal of a cell is below b, so
 * all points sharing a cell are pairwise linked (each cell is a clique).  A
 * linked pair is at most R = floor(b/w)+1 cells apart per dimension, so the
 * FoF components are the connected components of the cell graph whose edges
 * join cells (at offsets within +-R) that hold at least one linked pair.  The
 * occupied cells live in an open-addressing hash table.  Edge detection runs
 * in parallel (it only reads); the unions are applied sequentially. */
typedef struct {
    int64_t key;    /* linear cell id, -1 = empty slot */
    int64_t first;  /* offset of the cell's points in the bucketed order */
    int64_t count;
} slot_t;

static uint64_t mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

static int64_t hash_find(const slot_t *tab, uint64_t mask, int64_t key)
{
    uint64_t h = mix64((uint64_t)key) & mask;
    for (;;) {
        if (tab[h].key == key)
            return (int64_t)h;
        if (tab[h].key < 0)
            return -1;
        h = (h + 1) & mask;
    }
}

static int cmp_i64pair(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

int oracle_fof_cells(const float *xyz, int64_t n, double b, double b2, double L,
                     int32_t *labels, int nthreads)
{
    if (n < 1 || !(b > 0.0))
        return -1;
    set_threads(nthreads);
    double lo[3], hi[3];
    grid_box(xyz, n, L, lo, hi);
    grid_t g;
    g.L = L;
    const double w0 = b / sqrt(3.0) * (1.0 - 1e-9);
    double wmin = w0;
    for (int c = 0; c < 3; ++c) {
        g.lo[c] = lo[c];
        if (L > 0.0) {
            /* equal cells that tile the periodic side exactly */
            g.g[c] = (int64_t)ceil(L / w0);
            if (g.g[c] < 1) g.g[c] = 1;
            g.w[c] = L / (double)g.g[c];
        } else {
            g.w[c] = w0;
            g.g[c] = (int64_t)ceil((hi[c] - lo[c]) / w0) + 1; /* max may sit on the last face */
        }
        if (g.w[c] < wmin) wmin = g.w[c];
    }
    /* a linked pair is at most R cells apart in every dimension */
    const int64_t R = (int64_t)floor(b / wmin) + 1;
    const int64_t nnb = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    /* bucket points by cell: sort (cell id, index) pairs */
    int64_t *pairs = (int64_t *)malloc((size_t)n * 2 * sizeof(int64_t));
    if (!pairs)
        return -2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = cell_coord(&g, xyz[3 * i + 0], 0);
        int64_t cy = cell_coord(&g, xyz[3 * i + 1], 1);
        int64_t cz = cell_coord(&g, xyz[3 * i + 2], 2);
        pairs[2 * i] = (cx * g.g[1] + cy) * g.g[2] + cz;
        pairs[2 * i + 1] = i;
    }
    qsort(pairs, (size_t)n, 2 * sizeof(int64_t), cmp_i64pair);
    int64_t ncell = 0;
    for (int64_t t = 0; t < n; ++t)
        if (t == 0 || pairs[2 * t] != pairs[2 * t - 2])
            ++ncell;
    uint64_t cap = 1;
    while (cap < (uint64_t)ncell * 2)
        cap <<= 1;
    uint64_t mask = cap - 1;
    slot_t *tab = (slot_t *)malloc(cap * sizeof(slot_t));
    int64_t *cells = (int64_t *)malloc((size_t)ncell * sizeof(int64_t)); /* slot of each cell */
    int64_t *p = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!tab || !cells || !p) {
        free(pairs); free(tab); free(cells); free(p);
        return -2;
    }
    for (uint64_t h = 0; h < cap; ++h)
        tab[h].key = -1;
    {
        int64_t c = -1;
        for (int64_t t = 0; t < n; ++t) {
            int64_t key = pairs[2 * t];
            if (t == 0 || key != pairs[2 * t - 2]) {
                uint64_t h = mix64((uint64_t)key) & mask;
                while (tab[h].key >= 0)
                    h = (h + 1) & mask;
                tab[h].key = key;
                tab[h].first = t;
                tab[h].count = 0;
                cells[++c] = (int64_t)h;
            }
            tab[cells[c]].count++;
        }
    }
    /* union-find over points; first link each cell's clique to its smallest member
     * (the bucketed order keeps indices ascending within a cell) */
    for (int64_t i = 0; i < n; ++i)
        p[i] = i;
    for (int64_t c = 0; c < ncell; ++c) {
        const slot_t *s = &tab[cells[c]];
        int64_t head = pairs[2 * s->first + 1];
        for (int64_t t = 1; t < s->count; ++t)
            uf_union(p, head, pairs[2 * (s->first + t) + 1]);
    }
    /* cell-cell edges (each unordered pair once: the neighbour's key must be larger) */
    int nth = set_threads(0);
    int64_t **edges = (int64_t **)calloc((size_t)nth, sizeof(int64_t *));
    int64_t *ecount = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int64_t *ecap = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int failed = 0;
    int64_t **seenbuf = (int64_t **)calloc((size_t)nth, sizeof(int64_t *));
    for (int t = 0; t < nth; ++t) {
        seenbuf[t] = (int64_t *)malloc((size_t)nnb * sizeof(int64_t));
        if (!seenbuf[t])
            failed = 1;
    }
    if (failed) {
        for (int t = 0; t < nth; ++t)
            free(seenbuf[t]);
        free(seenbuf); free(edges); free(ecount); free(ecap);
        free(pairs); free(tab); free(cells); free(p);
        return -2;
    }
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 256)
        for (int64_t c = 0; c < ncell; ++c) {
            const slot_t *sa = &tab[cells[c]];
            int64_t key = sa->key;
            int64_t cz = key % g.g[2];
            int64_t cy = (key / g.g[2]) % g.g[1];
            int64_t cx = key / (g.g[2] * g.g[1]);
            int64_t *seen = seenbuf[tid];
            int64_t nseen = 0;
            for (int64_t dx = -R; dx <= R; ++dx)
                for (int64_t dy = -R; dy <= R; ++dy)
                    for (int64_t dz = -R; dz <= R; ++dz) {
                        int64_t o[3] = {cx + dx, cy + dy, cz + dz};
                        int ok = 1;
                        for (int d = 0; d < 3; ++d) {
                            if (L > 0.0)
                                o[d] = ((o[d] % g.g[d]) + g.g[d]) % g.g[d];
                            else if (o[d] < 0 || o[d] >= g.g[d])
                                ok = 0;
                        }
                        if (!ok)
                            continue;
                        int64_t nkey = (o[0] * g.g[1] + o[1]) * g.g[2] + o[2];
                        if (nkey <= key)
                            continue;
                        int dup = 0;
                        for (int64_t u = 0; u < nseen; ++u)
                            dup |= (seen[u] == nkey);
                        if (dup)
                            continue;
                        seen[nseen++] = nkey;
                        int64_t hb = hash_find(tab, mask, nkey);
                        if (hb < 0)
                            continue;
                        const slot_t *sb = &tab[hb];
                        int linked = 0;
                        for (int64_t ta = 0; ta < sa->count && !linked; ++ta) {
                            int64_t ia = pairs[2 * (sa->first + ta) + 1];
                            for (int64_t tb = 0; tb < sb->count; ++tb) {
                                int64_t ib = pairs[2 * (sb->first + tb) + 1];
                                if (pair_d2(xyz + 3 * ia, xyz + 3 * ib, L) <= b2) {
                                    linked = 1;
                                    break;
                                }
                            }
                        }
                        if (linked) {
                            if (ecount[tid] == ecap[tid]) {
                                int64_t nc = ecap[tid] ? 2 * ecap[tid] : 1024;
                                int64_t *ne = (int64_t *)realloc(edges[tid], (size_t)nc * 2 * sizeof(int64_t));
                                if (!ne) {
                                    failed = 1;
                                    continue;
                                }
                                edges[tid] = ne;
                                ecap[tid] = nc;
                            }
                            edges[tid][2 * ecount[tid]] = pairs[2 * sa->first + 1];
                            edges[tid][2 * ecount[tid] + 1] = pairs[2 * sb->first + 1];
                            ecount[tid]++;
                        }
                    }
        }
    }
    for (int t = 0; t < nth; ++t)
        free(seenbuf[t]);
    free(seenbuf);
    for (int t = 0; t < nth; ++t) {
        for (int64_t e = 0; e < ecount[t]; ++e)
            uf_union(p, edges[t][2 * e], edges[t][2 * e + 1]);
        free(edges[t]);
    }
    free(edges);
    free(ecount);
    free(ecap);
    for (int64_t i = 0; i < n; ++i)
        labels[i] = (int32_t)uf_find(p, i);
    free(pairs);
    free(tab);
    free(cells);
    free(p);
    return failed ? -2 : 0;
}
