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

/* kNN of separate query points among source points (Sec. II-G, multiple point
 * types): for query r, the k source points with the smallest (d2, source index). */
int oracle_knn_brute_sets(const float *src, int64_t n_src, const float *qry, int64_t n_qry, int k,
                          double L, int32_t *out_idx, double *out_d2, int nthreads)
{
    if (n_src < 1 || k < 1 || k > n_src || n_qry < 0)
        return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n_qry; ++r) {
        double *kd = out_d2 + r * k;
        int32_t *ki = out_idx + r * k;
        int m = 0;
        for (int64_t j = 0; j < n_src; ++j)
            topk_insert(kd, ki, &m, k, pair_d2(qry + 3 * r, src + 3 * j, L), (int32_t)j);
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
 * Cells of side w <= b_a/sqrt(3)*(1-1e-9): the diagonal of a cell is below b_a,
 * so all points sharing a cell are pairwise linked (each cell is a clique) for
 * both thresholds b2_a <= b2_b.  A pair within sqrt(b2_b) is at most
 * R = floor(sqrt(b2_b)/w) + 1 cells apart per dimension, so the FoF components of
 * each graph are the connected components of the cell graph whose edges join
 * cells (at offsets within +-R) holding at least one pair linked in that graph.
 * Points are bucketed by cell with an LSD radix sort of the cell keys; cells are
 * then grouped in rows of equal (cx, cy), and each row finds its neighbouring
 * rows once through a hash table of rows.  Edge detection runs in parallel over
 * rows (it only reads); the unions are applied sequentially. */
static uint64_t mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

typedef struct {
    int64_t key;    /* row id cx*gy + cy, -1 = empty slot */
    int64_t first;  /* first cell of the row */
    int64_t last;   /* one past the last cell */
} row_slot_t;

static int64_t row_find(const row_slot_t *tab, uint64_t mask, int64_t key)
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

/* stable LSD radix sort of (key, index) pairs on the low `bits` bits */
static int radix_pairs(int64_t *key, int64_t *idx, int64_t n, int bits)
{
    int64_t *k2 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *i2 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *cnt = (int64_t *)malloc((1 << 16) * sizeof(int64_t));
    if (!k2 || !i2 || !cnt) {
        free(k2); free(i2); free(cnt);
        return -2;
    }
    for (int sh = 0; sh < bits; sh += 16) {
        memset(cnt, 0, (1 << 16) * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i)
            cnt[((uint64_t)key[i] >> sh) & 0xffff]++;
        int64_t run = 0;
        for (int d = 0; d < (1 << 16); ++d) {
            int64_t c = cnt[d];
            cnt[d] = run;
            run += c;
        }
        for (int64_t i = 0; i < n; ++i) {
            int64_t pos = cnt[((uint64_t)key[i] >> sh) & 0xffff]++;
            k2[pos] = key[i];
            i2[pos] = idx[i];
        }
        memcpy(key, k2, (size_t)n * sizeof(int64_t));
        memcpy(idx, i2, (size_t)n * sizeof(int64_t));
    }
    free(k2); free(i2); free(cnt);
    return 0;
}

typedef struct {
    int64_t *e;   /* pairs (a, b, flag) */
    int64_t n, cap;
} edges_t;

static int edge_push(edges_t *E, int64_t a, int64_t b, int64_t flag)
{
    if (E->n == E->cap) {
        int64_t nc = E->cap ? 2 * E->cap : 4096;
        int64_t *ne = (int64_t *)realloc(E->e, (size_t)nc * 3 * sizeof(int64_t));
        if (!ne)
            return -2;
        E->e = ne;
        E->cap = nc;
    }
    E->e[3 * E->n] = a;
    E->e[3 * E->n + 1] = b;
    E->e[3 * E->n + 2] = flag;
    E->n++;
    return 0;
}

/* labels_a: FoF at b2_a, labels_b: FoF at b2_b (b2_a <= b2_b); labels_b may be NULL */
int oracle_fof_cells2(const float *xyz, int64_t n, double b2_a, double b2_b, double L,
                      int32_t *labels_a, int32_t *labels_b, int nthreads)
{
    if (n < 1 || !(b2_a > 0.0) || b2_b < b2_a)
        return -1;
    set_threads(nthreads);
    double lo[3], hi[3];
    grid_box(xyz, n, L, lo, hi);
    grid_t g;
    g.L = L;
    const double w0 = sqrt(b2_a) / sqrt(3.0) * (1.0 - 1e-9);
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
    const int64_t R = (int64_t)floor(sqrt(b2_b) / wmin) + 1;
    int key_bits = 0;
    while (key_bits < 63 && ((uint64_t)1 << key_bits) < (uint64_t)(g.g[0] * g.g[1] * g.g[2]))
        ++key_bits;
    int64_t *key = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *pt = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *p = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *q = labels_b ? (int64_t *)malloc((size_t)n * sizeof(int64_t)) : NULL;
    if (!key || !pt || !p || (labels_b && !q)) {
        free(key); free(pt); free(p); free(q);
        return -2;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = cell_coord(&g, xyz[3 * i + 0], 0);
        int64_t cy = cell_coord(&g, xyz[3 * i + 1], 1);
        int64_t cz = cell_coord(&g, xyz[3 * i + 2], 2);
        key[i] = (cx * g.g[1] + cy) * g.g[2] + cz;
        pt[i] = i;
    }
    if (radix_pairs(key, pt, n, key_bits)) {
        free(key); free(pt); free(p); free(q);
        return -2;
    }
    /* cells (runs of equal keys) and rows (runs of equal key / gz) */
    int64_t ncell = 0, nrow = 0;
    for (int64_t t = 0; t < n; ++t) {
        if (t == 0 || key[t] != key[t - 1]) ++ncell;
        if (t == 0 || key[t] / g.g[2] != key[t - 1] / g.g[2]) ++nrow;
    }
    int64_t *cfirst = (int64_t *)malloc((size_t)(ncell + 1) * sizeof(int64_t));
    int64_t *ckey = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    int64_t *rcell = (int64_t *)malloc((size_t)(nrow + 1) * sizeof(int64_t));
    uint64_t cap = 1;
    while (cap < (uint64_t)nrow * 2) cap <<= 1;
    const uint64_t mask = cap - 1;
    row_slot_t *rows = (row_slot_t *)malloc(cap * sizeof(row_slot_t));
    if (!cfirst || !ckey || !rcell || !rows) {
        free(key); free(pt); free(p); free(q); free(cfirst); free(ckey); free(rcell); free(rows);
        return -2;
    }
    {
        int64_t c = -1, r = -1;
        for (int64_t t = 0; t < n; ++t) {
            if (t == 0 || key[t] != key[t - 1]) {
                ++c;
                cfirst[c] = t;
                ckey[c] = key[t];
                if (c == 0 || ckey[c] / g.g[2] != ckey[c - 1] / g.g[2])
                    rcell[++r] = c;
            }
        }
        cfirst[ncell] = n;
        rcell[nrow] = ncell;
    }
    for (uint64_t h = 0; h < cap; ++h)
        rows[h].key = -1;
    for (int64_t r = 0; r < nrow; ++r) {
        int64_t rk = ckey[rcell[r]] / g.g[2];
        uint64_t h = mix64((uint64_t)rk) & mask;
        while (rows[h].key >= 0)
            h = (h + 1) & mask;
        rows[h].key = rk;
        rows[h].first = rcell[r];
        rows[h].last = rcell[r + 1];
    }
    /* union-find; first link each cell's clique to its first member */
    for (int64_t i = 0; i < n; ++i) {
        p[i] = i;
        if (q) q[i] = i;
    }
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t head = pt[cfirst[c]];
        for (int64_t t = cfirst[c] + 1; t < cfirst[c + 1]; ++t) {
            uf_union(p, head, pt[t]);
            if (q) uf_union(q, head, pt[t]);
        }
    }
    int nth = set_threads(0);
    edges_t *E = (edges_t *)calloc((size_t)nth, sizeof(edges_t));
    int failed = 0;
    const int64_t nnb = (2 * R + 1) * (2 * R + 1);
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t *nb_first = (int64_t *)malloc((size_t)nnb * sizeof(int64_t));
        int64_t *nb_last = (int64_t *)malloc((size_t)nnb * sizeof(int64_t));
        int64_t *nb_row = (int64_t *)malloc((size_t)nnb * sizeof(int64_t));
        if (!nb_first || !nb_last || !nb_row)
            failed = 1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nrow; ++r) {
            if (failed)
                continue;
            const int64_t rk = ckey[rcell[r]] / g.g[2];
            const int64_t cx = rk / g.g[1], cy = rk % g.g[1];
            /* neighbouring rows, each once (periodic wrap may repeat them) */
            int64_t nn = 0;
            for (int64_t dx = -R; dx <= R; ++dx)
                for (int64_t dy = -R; dy <= R; ++dy) {
                    int64_t ox = cx + dx, oy = cy + dy;
                    if (L > 0.0) {
                        ox = ((ox % g.g[0]) + g.g[0]) % g.g[0];
                        oy = ((oy % g.g[1]) + g.g[1]) % g.g[1];
                    } else if (ox < 0 || ox >= g.g[0] || oy < 0 || oy >= g.g[1]) {
                        continue;
                    }
                    int64_t ork = ox * g.g[1] + oy;
                    int dup = 0;
                    for (int64_t u = 0; u < nn; ++u)
                        dup |= (nb_row[u] == ork);
                    if (dup)
                        continue;
                    int64_t h = row_find(rows, mask, ork);
                    if (h < 0)
                        continue;
                    nb_row[nn] = ork;
                    nb_first[nn] = rows[h].first;
                    nb_last[nn] = rows[h].last;
                    ++nn;
                }
            for (int64_t ca = rcell[r]; ca < rcell[r + 1]; ++ca) {
                const int64_t cz = ckey[ca] % g.g[2];
                for (int64_t u = 0; u < nn; ++u) {
                    for (int64_t cb = nb_first[u]; cb < nb_last[u]; ++cb) {
                        if (ckey[cb] <= ckey[ca])
                            continue; /* each unordered cell pair once */
                        int64_t dz = ckey[cb] % g.g[2] - cz;
                        if (L > 0.0) {
                            dz = ((dz % g.g[2]) + g.g[2]) % g.g[2];
                            if (dz > g.g[2] - dz) dz = g.g[2] - dz;
                        } else if (dz < 0) {
                            dz = -dz;
                        }
                        if (dz > R)
                            continue;
                        int la = 0, lb = 0;
                        for (int64_t ta = cfirst[ca]; ta < cfirst[ca + 1] && !la; ++ta) {
                            const int64_t ia = pt[ta];
                            for (int64_t tb = cfirst[cb]; tb < cfirst[cb + 1]; ++tb) {
                                const double d2 = pair_d2(xyz + 3 * ia, xyz + 3 * pt[tb], L);
                                if (d2 <= b2_a) {
                                    la = 1;
                                    break;
                                }
                                if (d2 <= b2_b)
                                    lb = 1;
                            }
                        }
                        if ((la || lb) && edge_push(&E[tid], pt[cfirst[ca]], pt[cfirst[cb]], la))
                            failed = 1;
                    }
                }
            }
        }
        free(nb_first);
        free(nb_last);
        free(nb_row);
    }
    for (int t = 0; t < nth; ++t) {
        for (int64_t e = 0; e < E[t].n; ++e) {
            const int64_t a = E[t].e[3 * e], b = E[t].e[3 * e + 1];
            if (E[t].e[3 * e + 2])
                uf_union(p, a, b);
            if (q)
                uf_union(q, a, b);
        }
        free(E[t].e);
    }
    free(E);
    for (int64_t i = 0; i < n; ++i) {
        labels_a[i] = (int32_t)uf_find(p, i);
        if (q) labels_b[i] = (int32_t)uf_find(q, i);
    }
    free(key); free(pt); free(p); free(q); free(cfirst); free(ckey); free(rcell); free(rows);
    return failed ? -2 : 0;
}

int oracle_fof_cells(const float *xyz, int64_t n, double b, double b2, double L,
                     int32_t *labels, int nthreads)
{
    (void)b;
    return oracle_fof_cells2(xyz, n, b2, b2, L, labels, NULL, nthreads);
}
