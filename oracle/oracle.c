/*
 * oracle.c -- plain, slow, FP64 CPU restatement of the graph-construction
 * path of "Revisiting the Index Construction of Proximity Graph-Based
 * Approximate Nearest Neighbor Search" (arXiv 2410.01231).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check
 * and the benchmark's CPU-baseline leg may load this library.  The product
 * (the CUDA library) shares no code with it and never calls it.
 *
 * Arithmetic rules (fixed so that a GPU FP64 recheck can reproduce any
 * single value bit for bit):
 *   - every distance is accumulated in double, sequentially in coordinate
 *     order, one rounding per multiply and per add (build with
 *     -ffp-contract=off; no fused multiply-add);
 *   - square roots are IEEE sqrt();
 *   - cos(alpha) is supplied by the caller as a double.
 * Orders are always by the pair (distance, id), ascending.
 *
 * Which passage each function follows is stated above it.  Where the paper
 * is silent the reading taken is stated as well.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_L2SQ = 0, OR_COSINE = 1, OR_IP = 2 };

/* ---------------------------------------------------------------------- */
/* Distances.  Section 2: dist(u,v) is the Euclidean (L2) norm; ranking by */
/* its square is the same ranking.  Reading for unit-norm data (cosine and */
/* inner product): s = 2 - 2<x,y>, the squared chord, clamped at 0, which  */
/* equals squared L2 on the unit sphere and orders like -<x,y>.            */
/* ---------------------------------------------------------------------- */
double or_dist(const float *x, const float *y, int d, int metric)
{
    double s = 0.0;
    if (metric == OR_L2SQ) {
        for (int i = 0; i < d; ++i) {
            double t = (double)x[i] - (double)y[i];
            s = s + t * t;
        }
        return s;
    }
    for (int i = 0; i < d; ++i)
        s = s + (double)x[i] * (double)y[i];
    s = 2.0 - 2.0 * s;
    return s < 0.0 ? 0.0 : s;
}

/* distance between a float row and a double point (used for the centroid) */
static double dist_to_point(const float *x, const double *c, int d, int metric)
{
    double s = 0.0;
    if (metric == OR_L2SQ) {
        for (int i = 0; i < d; ++i) {
            double t = (double)x[i] - c[i];
            s = s + t * t;
        }
        return s;
    }
    for (int i = 0; i < d; ++i)
        s = s + (double)x[i] * c[i];
    s = 2.0 - 2.0 * s;
    return s < 0.0 ? 0.0 : s;
}

typedef struct {
    double s;
    int32_t id;
} item_t;

static int item_less(item_t a, item_t b)
{
    return a.s < b.s || (a.s == b.s && a.id < b.id);
}

static int item_cmp(const void *pa, const void *pb)
{
    item_t a = *(const item_t *)pa, b = *(const item_t *)pb;
    if (item_less(a, b)) return -1;
    if (item_less(b, a)) return 1;
    return 0;
}

/* keep the `cap` smallest items of a stream: sorted insertion */
static int topk_push(item_t *top, int cnt, int cap, item_t it)
{
    if (cnt == cap && !item_less(it, top[cap - 1]))
        return cnt;
    int j = cnt < cap ? cnt : cap - 1;
    while (j > 0 && item_less(it, top[j - 1])) {
        top[j] = top[j - 1];
        --j;
    }
    top[j] = it;
    return cnt < cap ? cnt + 1 : cnt;
}

/* ---------------------------------------------------------------------- */
/* Exact k-nearest neighbours (the KNNG of the initialization phase,      */
/* Section 3.1 / Algorithm 6, computed exactly by brute force).           */
/* For query row q the K smallest (s(q,v), v) over all v != exclude[q].    */
/* Q may be D itself (exclude[q] = q) or external queries (exclude NULL). */
/* Rows shorter than K (n-1 < K) are padded with id -1, dist +inf.        */
/* ---------------------------------------------------------------------- */
int or_knn(const float *D, int64_t n, int d, int metric, const float *Q, int64_t nq,
           const int64_t *exclude, int K, int32_t *ids, double *dist)
{
    int bad = 0;
#pragma omp parallel
    {
        item_t *top = (item_t *)malloc(sizeof(item_t) * (size_t)K);
        if (!top) bad = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < nq; ++q) {
            if (!top) continue;
            int cnt = 0;
            const float *x = Q + (size_t)q * d;
            int64_t ex = exclude ? exclude[q] : -1;
            for (int64_t v = 0; v < n; ++v) {
                if (v == ex) continue;
                item_t it = { or_dist(x, D + (size_t)v * d, d, metric), (int32_t)v };
                cnt = topk_push(top, cnt, K, it);
            }
            for (int j = 0; j < K; ++j) {
                ids[q * K + j] = j < cnt ? top[j].id : -1;
                dist[q * K + j] = j < cnt ? top[j].s : INFINITY;
            }
        }
        free(top);
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* alpha-pruning (Section 4.1 definition) applied in the scan order of    */
/* Prune, Algorithm 3.                                                     */
/*                                                                        */
/* Candidates are taken in ascending (s(u,v), v) order after dropping u    */
/* itself, negative ids and repeated ids.  v is occluded by an already     */
/* kept w iff                                                              */
/*      s(u,w) < s(u,v)  and  s(v,w) < s(u,v)  and  angle(u,w,v) > alpha.  */
/* Reading: both distance inequalities strict, as in the RNG and alpha-    */
/* pruning definitions (Section 2.1, Section 4.1).  With s = squared L2 the */
/* angle at w satisfies, by the law of cosines,                            */
/*      cos(angle) = (s(u,w) + s(v,w) - s(u,v)) / (2 sqrt(s(u,w) s(v,w))), */
/* so "angle > alpha" is  s(u,w)+s(v,w)-s(u,v) < 2 cos(alpha) sqrt(s(u,w) s(v,w)). */
/* alpha = 60 degrees is RNG pruning exactly (Section 4.2): when uv is the */
/* strictly longest side of the triangle its opposite angle exceeds 60,   */
/* so with alpha60 set the angle clause is skipped.                        */
/* The scan stops once R candidates are kept (Algorithm 3).               */
/* Returns the number kept; out[] receives them in scan order.            */
/* ---------------------------------------------------------------------- */
static int angle_exceeds(double suw, double svw, double suv, double cos_alpha)
{
    double lhs = (suw + svw) - suv;
    double rhs = (2.0 * cos_alpha) * sqrt(suw * svw);
    return lhs < rhs;
}

static int prune_one(const float *D, int d, int metric, int64_t u, const int32_t *cand,
                     int64_t nc, int R, double cos_alpha, int alpha60, item_t *buf,
                     int32_t *out, double *out_s)
{
    const float *xu = D + (size_t)u * d;
    int64_t m = 0;
    for (int64_t j = 0; j < nc; ++j) {
        int32_t v = cand[j];
        if (v < 0 || v == u) continue;
        buf[m].s = or_dist(xu, D + (size_t)v * d, d, metric);
        buf[m].id = v;
        ++m;
    }
    qsort(buf, (size_t)m, sizeof(item_t), item_cmp);
    int kept = 0;
    for (int64_t j = 0; j < m && kept < R; ++j) {
        if (j > 0 && buf[j].id == buf[j - 1].id) continue; /* repeated id */
        int32_t v = buf[j].id;
        double suv = buf[j].s;
        const float *xv = D + (size_t)v * d;
        int occluded = 0;
        for (int t = 0; t < kept && !occluded; ++t) {
            double suw = out_s[t];
            if (!(suw < suv)) continue;
            double svw = or_dist(xv, D + (size_t)out[t] * d, d, metric);
            if (!(svw < suv)) continue;
            if (alpha60 || angle_exceeds(suw, svw, suv, cos_alpha)) occluded = 1;
        }
        if (!occluded) {
            out[kept] = v;
            out_s[kept] = suv;
            ++kept;
        }
    }
    return kept;
}

/* Prune every row of a CSR candidate set.  nbr is [n][R] (-1 padded). */
int or_prune(const float *D, int64_t n, int d, int metric, const int64_t *off,
             const int32_t *cand, int R, double cos_alpha, int alpha60, int32_t *nbr,
             int32_t *deg)
{
    int64_t maxc = 0;
    for (int64_t u = 0; u < n; ++u)
        if (off[u + 1] - off[u] > maxc) maxc = off[u + 1] - off[u];
    int bad = 0;
#pragma omp parallel
    {
        item_t *buf = (item_t *)malloc(sizeof(item_t) * (size_t)(maxc + 1));
        int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
        double *out_s = (double *)malloc(sizeof(double) * (size_t)R);
        if (!buf || !out || !out_s) bad = 1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < n; ++u) {
            if (bad) continue;
            int k = prune_one(D, d, metric, u, cand + off[u], off[u + 1] - off[u], R,
                              cos_alpha, alpha60, buf, out, out_s);
            for (int j = 0; j < R; ++j) nbr[u * R + j] = j < k ? out[j] : -1;
            deg[u] = k;
        }
        free(buf);
        free(out);
        free(out_s);
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Reverse-edge union (Algorithm 2; Algorithm 5):                         */
/* row u of the result is N(u) followed by every v with u in N(v), v in   */
/* increasing order.  Every row reads the same input graph (the pass-1    */
/* lists), our reading of a step the paper runs for all u at once.  Then */
/* Prune sorts and de-duplicates.  off has n+1 entries; ids needs off[n] */
/* slots: call with ids == NULL to get the total.                         */
/* ---------------------------------------------------------------------- */
int64_t or_reverse_union(const int32_t *nbr, const int32_t *deg, int64_t n, int R,
                         int64_t *off, int32_t *ids)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t v = 0; v < n; ++v) {
        cnt[v] += deg[v];
        for (int j = 0; j < deg[v]; ++j) cnt[nbr[v * R + j]] += 1;
    }
    off[0] = 0;
    for (int64_t u = 0; u < n; ++u) off[u + 1] = off[u] + cnt[u];
    if (ids) {
        int64_t *pos = cnt; /* reuse as the fill cursor */
        for (int64_t u = 0; u < n; ++u) {
            pos[u] = off[u];
            for (int j = 0; j < deg[u]; ++j) ids[pos[u]++] = nbr[u * R + j];
        }
        for (int64_t v = 0; v < n; ++v)
            for (int j = 0; j < deg[v]; ++j) {
                int64_t u = nbr[v * R + j];
                ids[pos[u]++] = (int32_t)v;
            }
    }
    free(cnt);
    return off[n];
}

/* ---------------------------------------------------------------------- */
/* Entry point: the point closest to the centroid of D (Section 3.1,     */
/* search phase, which names this point as the entry).  Reading:          */
/* the exact argmin over all points, ties by id.  The centroid is summed  */
/* in double per coordinate in blocks of 1024 consecutive points (each    */
/* block summed in index order, then the block sums added in block order) */
/* and divided by n.                                                       */
/* ---------------------------------------------------------------------- */
#define OR_CENTROID_BLOCK 1024

int64_t or_medoid(const float *D, int64_t n, int d, int metric, double *centroid_out)
{
    double *c = (double *)calloc((size_t)d, sizeof(double));
    if (!c || n <= 0) {
        free(c);
        return -1;
    }
    for (int i = 0; i < d; ++i) {
        double total = 0.0;
        for (int64_t b = 0; b < n; b += OR_CENTROID_BLOCK) {
            double part = 0.0;
            int64_t e = b + OR_CENTROID_BLOCK < n ? b + OR_CENTROID_BLOCK : n;
            for (int64_t v = b; v < e; ++v) part = part + (double)D[v * d + i];
            total = total + part;
        }
        c[i] = total / (double)n;
    }
    item_t best = { INFINITY, -1 };
    for (int64_t v = 0; v < n; ++v) {
        item_t it = { dist_to_point(D + (size_t)v * d, c, d, metric), (int32_t)v };
        if (best.id < 0 || item_less(it, best)) best = it;
    }
    if (centroid_out) memcpy(centroid_out, c, sizeof(double) * (size_t)d);
    free(c);
    return best.id;
}

/* ---------------------------------------------------------------------- */
/* Connectivity (Algorithm 2; Algorithm 5).  The paper finds connected  */
/* components by depth-first search and links them with extra edges.     */
/* Reading,                                                               */
/* deterministic: S = nodes reachable from ep along directed edges.  While */
/* S != V: r = smallest unreached id; p = argmin over x in S with          */
/* deg(x) < R of (s(x,r), x); append r to N(p); add everything reachable  */
/* from r to S.  The search order of the reachability pass does not change */
/* S, so a breadth-first queue is used.  Returns the number of edges      */
/* added, or -1 when no reached node has a free slot (the library reports */
/* the same case as an error).                                             */
/* ---------------------------------------------------------------------- */
static int64_t reach_from(const int32_t *nbr, const int32_t *deg, int R, int64_t src,
                          uint8_t *inS, int64_t *queue)
{
    int64_t head = 0, tail = 0, added = 0;
    if (inS[src]) return 0;
    inS[src] = 1;
    queue[tail++] = src;
    ++added;
    while (head < tail) {
        int64_t x = queue[head++];
        for (int j = 0; j < deg[x]; ++j) {
            int64_t y = nbr[x * R + j];
            if (!inS[y]) {
                inS[y] = 1;
                queue[tail++] = y;
                ++added;
            }
        }
    }
    return added;
}

/* The nearest reached node with a free slot to the row xr: argmin over  */
/* x with inS[x] and deg[x] < R of the pair (s(x, r), x).  The minimum of  */
/* a total order does not depend on how the scan is split among threads.   */
static item_t nearest_reached_free(const float *D, int64_t n, int d, int metric,
                                   const uint8_t *inS, const int32_t *deg, int R, const float *xr)
{
    item_t best = { INFINITY, -1 };
#pragma omp parallel
    {
        item_t loc = { INFINITY, -1 };
#pragma omp for schedule(static)
        for (int64_t x = 0; x < n; ++x) {
            if (!inS[x] || deg[x] >= R) continue;
            item_t it = { or_dist(D + (size_t)x * d, xr, d, metric), (int32_t)x };
            if (loc.id < 0 || item_less(it, loc)) loc = it;
        }
#pragma omp critical
        {
            if (loc.id >= 0 && (best.id < 0 || item_less(loc, best))) best = loc;
        }
    }
    return best;
}

int64_t or_connect(const float *D, int64_t n, int d, int metric, int32_t *nbr, int32_t *deg,
                   int R, int64_t ep)
{
    uint8_t *inS = (uint8_t *)calloc((size_t)n, 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!inS || !queue) {
        free(inS);
        free(queue);
        return -2;
    }
    int64_t reached = reach_from(nbr, deg, R, ep, inS, queue);
    int64_t edges = 0, r = 0;
    while (reached < n) {
        while (inS[r]) ++r;
        const float *xr = D + (size_t)r * d;
        item_t best = nearest_reached_free(D, n, d, metric, inS, deg, R, xr);
        if (best.id < 0) {
            edges = -1;
            break;
        }
        nbr[(int64_t)best.id * R + deg[best.id]] = (int32_t)r;
        deg[best.id] += 1;
        ++edges;
        reached += reach_from(nbr, deg, R, r, inS, queue);
    }
    free(inS);
    free(queue);
    return edges;
}

/* ---------------------------------------------------------------------- */
/* The connectivity step with edge replacement (a reading for graphs whose */
/* reached nodes are all full, not used by the builds): as or_connect, but */
/* when no reached node has a free slot, the reached node p nearest to r   */
/* that still holds an edge not added by this step gives up the last such */
/* edge in its list (its farthest original neighbour) for r, and the      */
/* reached set is recomputed from ep, since the dropped edge may have been */
/* the only route to some nodes (p itself stays reached: a route to p     */
/* never needs p's own out-edges).  Every replacement removes one original */
/* edge and every free-slot link grows the reached set, so the loop ends. */
/* Returns the edges added (replacements included; *replaced counts them), */
/* -1 when no reached node has a free slot or an original edge.           */
/* ---------------------------------------------------------------------- */
int64_t or_connect_replace(const float *D, int64_t n, int d, int metric, int32_t *nbr,
                           int32_t *deg, int R, int64_t ep, int64_t *replaced)
{
    uint8_t *inS = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *added_here = (uint8_t *)calloc((size_t)(n * R), 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!inS || !added_here || !queue) {
        free(inS);
        free(added_here);
        free(queue);
        return -2;
    }
    int64_t reached = reach_from(nbr, deg, R, ep, inS, queue);
    int64_t edges = 0, rep = 0, r = 0;
    while (reached < n) {
        while (inS[r]) ++r;
        const float *xr = D + (size_t)r * d;
        item_t best = nearest_reached_free(D, n, d, metric, inS, deg, R, xr);
        if (best.id >= 0) {
            added_here[(int64_t)best.id * R + deg[best.id]] = 1;
            nbr[(int64_t)best.id * R + deg[best.id]] = (int32_t)r;
            deg[best.id] += 1;
            ++edges;
            reached += reach_from(nbr, deg, R, r, inS, queue);
            continue;
        }
        for (int64_t x = 0; x < n; ++x) {
            if (!inS[x]) continue;
            int has = 0;
            for (int j = 0; j < deg[x] && !has; ++j) has = !added_here[x * R + j];
            if (!has) continue;
            item_t it = { or_dist(D + (size_t)x * d, xr, d, metric), (int32_t)x };
            if (best.id < 0 || item_less(it, best)) best = it;
        }
        if (best.id < 0) {
            edges = -1;
            break;
        }
        const int64_t p = best.id;
        int slot = deg[p] - 1;
        while (added_here[p * R + slot]) --slot;
        nbr[p * R + slot] = (int32_t)r;
        added_here[p * R + slot] = 1;
        ++edges;
        ++rep;
        memset(inS, 0, (size_t)n);
        reached = reach_from(nbr, deg, R, ep, inS, queue);
        r = 0;
    }
    if (replaced) *replaced = rep;
    free(inS);
    free(added_here);
    free(queue);
    return edges;
}

/* ---------------------------------------------------------------------- */
/* Beam search, KANNSearch(G, q, k, L, ep) of Algorithm 1.                 */
/*                                                                        */
/* pool: at most L (s, id, expanded) entries sorted by (s, id).  It starts */
/* with the entry point(s).  Repeat: take the first unexpanded entry among */
/* pool[0 .. min(L,|pool|)-1] (none left: stop), mark it expanded, insert  */
/* each of its out-neighbours with its distance, sort, keep the first L.  */
/* Return pool[0 .. k-1].                                                  */
/* Readings where the paper is silent: a shorter pool counts as fully     */
/* expanded; a node is inserted at most once per search (policy 0 keeps an */
/* exact visited set).  policy 1 only refuses ids already in the pool:    */
/* since the pool is always the L best of everything inserted so far, a   */
/* node that left it can never re-enter, so both policies return the same */
/* pool (the tests check this).                                            */
/* rows: optional map id -> adjacency row (for the layers of a            */
/* hierarchical graph whose rows are a subset); NULL means row = id.      */
/* ---------------------------------------------------------------------- */
typedef struct {
    double s;
    int32_t id;
    int32_t expanded;
} pent_t;

static int pent_cmp(const void *pa, const void *pb)
{
    const pent_t *a = (const pent_t *)pa, *b = (const pent_t *)pb;
    if (a->s < b->s || (a->s == b->s && a->id < b->id)) return -1;
    if (b->s < a->s || (b->s == a->s && b->id < a->id)) return 1;
    return 0;
}

static int search_one(const float *D, int d, int metric, const int32_t *nbr,
                      const int32_t *deg, int R, const int32_t *rows, const float *q,
                      const int32_t *starts, int nstarts, int L, int policy, int32_t *stamp,
                      int32_t mark, pent_t *pool, int64_t *n_expanded)
{
    int size = 0;
    for (int t = 0; t < nstarts; ++t) {
        int32_t e = starts[t];
        if (e < 0 || stamp[e] == mark) continue;
        stamp[e] = mark;
        pool[size].s = or_dist(q, D + (size_t)e * d, d, metric);
        pool[size].id = e;
        pool[size].expanded = 0;
        ++size;
    }
    qsort(pool, (size_t)size, sizeof(pent_t), pent_cmp);
    if (size > L) size = L;
    for (;;) {
        int i = 0;
        while (i < size && pool[i].expanded) ++i;
        if (i >= size) break;
        pool[i].expanded = 1;
        if (n_expanded) ++*n_expanded;
        int64_t row = rows ? rows[pool[i].id] : pool[i].id;
        int m = size;
        for (int j = 0; j < deg[row]; ++j) {
            int32_t v = nbr[row * R + j];
            if (policy == 0) {
                if (stamp[v] == mark) continue;
                stamp[v] = mark;
            } else {
                int dup = 0;
                for (int t = 0; t < m; ++t)
                    if (pool[t].id == v) dup = 1;
                if (dup) continue;
            }
            pool[m].s = or_dist(q, D + (size_t)v * d, d, metric);
            pool[m].id = v;
            pool[m].expanded = 0;
            ++m;
        }
        qsort(pool, (size_t)m, sizeof(pent_t), pent_cmp);
        size = m < L ? m : L;
    }
    return size;
}

/* Batched queries.  starts: nq x nstarts entry points (row-major).        */
/* Output rows of k, padded with -1 / +inf.                                */
int or_search(const float *D, int64_t n, int d, int metric, const int32_t *nbr,
              const int32_t *deg, int R, const int32_t *rows, const float *Q, int64_t nq,
              const int32_t *starts, int nstarts, int k, int L, int policy, int32_t *out_ids,
              double *out_dist, int64_t *n_expanded)
{
    int bad = 0;
    int64_t expanded_total = 0;
#pragma omp parallel reduction(+ : expanded_total)
    {
        int32_t *stamp = (int32_t *)calloc((size_t)n, sizeof(int32_t));
        pent_t *pool = (pent_t *)malloc(sizeof(pent_t) * (size_t)(L + R + nstarts + 1));
        if (!stamp || !pool) bad = 1;
        int32_t mark = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t qi = 0; qi < nq; ++qi) {
            if (!stamp || !pool) continue;
            ++mark;
            int64_t ne = 0;
            int size = search_one(D, d, metric, nbr, deg, R, rows, Q + (size_t)qi * d,
                                  starts + qi * nstarts, nstarts, L, policy, stamp, mark,
                                  pool, &ne);
            expanded_total += ne;
            for (int j = 0; j < k; ++j) {
                out_ids[qi * k + j] = j < size ? pool[j].id : -1;
                out_dist[qi * k + j] = j < size ? pool[j].s : INFINITY;
            }
        }
        free(stamp);
        free(pool);
    }
    if (n_expanded) *n_expanded = expanded_total;
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* k-CNA by search on the refined graph (Algorithm 5):                    */
/* C(u) <- KANNSearch(G^, u, L, L, u): every point searches for itself,    */
/* starting at itself, with pool width L.  The row keeps the pool minus u */
/* itself, in pool order, padded with -1 to L entries.                     */
/* ---------------------------------------------------------------------- */
int or_acquire(const float *D, int64_t n, int d, int metric, const int32_t *nbr,
               const int32_t *deg, int R, int L, int32_t *cand, int64_t *n_expanded)
{
    int bad = 0;
    int64_t expanded_total = 0;
#pragma omp parallel reduction(+ : expanded_total)
    {
        int32_t *stamp = (int32_t *)calloc((size_t)n, sizeof(int32_t));
        pent_t *pool = (pent_t *)malloc(sizeof(pent_t) * (size_t)(L + R + 2));
        if (!stamp || !pool) bad = 1;
        int32_t mark = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t u = 0; u < n; ++u) {
            if (!stamp || !pool) continue;
            ++mark;
            int32_t start = (int32_t)u;
            int64_t ne = 0;
            int size = search_one(D, d, metric, nbr, deg, R, NULL, D + (size_t)u * d, &start, 1,
                                  L, 0, stamp, mark, pool, &ne);
            expanded_total += ne;
            int w = 0;
            for (int j = 0; j < size; ++j)
                if (pool[j].id != u) cand[u * L + w++] = pool[j].id;
            while (w < L) cand[u * L + w++] = -1;
        }
        free(stamp);
        free(pool);
    }
    if (n_expanded) *n_expanded = expanded_total;
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* IterNSG with a fixed number of iterations (Algorithm 6; I = 2 is the   */
/* paper's default, Exp.1-a), each iteration being OptKCNA (Algorithm 5): */
/*   C(u) <- kNN row of u                                                  */
/*   repeat I times:                                                       */
/*     N <- Prune(C, R, alpha);  N <- Prune(N u reverse(N), R, alpha);     */
/*     connect(N, ep);  C(u) <- KANNSearch(N, u, L, L, u)                  */
/*   final Refine (Algorithm 2): the same two prunes with                 */
/*   alpha = alpha_final (60 degrees: RNG pruning), then connect unless    */
/*   connect_final is 0 (NSWG layers, Section 5.3).                        */
/* ep is the medoid (or_medoid).  Outputs nbr [n][R], deg [n]; returns ep, */
/* or a negative value on failure (-1: connect found no free slot).        */
/* cos_alpha values come from the caller.                                   */
/* ---------------------------------------------------------------------- */
static int refine(const float *D, int64_t n, int d, int metric, const int64_t *off,
                  const int32_t *cand, int R, double cos_a, int a60, int32_t *nbr,
                  int32_t *deg, int do_connect, int64_t ep)
{
    int32_t *tmp_nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * R));
    int32_t *tmp_deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *uoff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int rc = 0;
    if (!tmp_nbr || !tmp_deg || !uoff) rc = -2;
    if (!rc) rc = or_prune(D, n, d, metric, off, cand, R, cos_a, a60, tmp_nbr, tmp_deg);
    int32_t *uids = NULL;
    if (!rc) {
        int64_t tot = or_reverse_union(tmp_nbr, tmp_deg, n, R, uoff, NULL);
        uids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot + 1));
        if (!uids) rc = -2;
        else or_reverse_union(tmp_nbr, tmp_deg, n, R, uoff, uids);
    }
    if (!rc) rc = or_prune(D, n, d, metric, uoff, uids, R, cos_a, a60, nbr, deg);
    if (!rc && do_connect && or_connect(D, n, d, metric, nbr, deg, R, ep) < 0) rc = -1;
    free(tmp_nbr);
    free(tmp_deg);
    free(uoff);
    free(uids);
    return rc;
}

int64_t or_build_rng(const float *D, int64_t n, int d, int metric, int K, int L, int R,
                     double cos_alpha, int alpha60, double cos_alpha_final, int alpha_final60,
                     int iters, int connect_final, int32_t *nbr, int32_t *deg)
{
    if (n < 2) return -3;
    int Kc = K < n - 1 ? K : (int)(n - 1);
    int64_t ep = or_medoid(D, n, d, metric, NULL);
    int32_t *knn_ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * Kc));
    double *knn_d = (double *)malloc(sizeof(double) * (size_t)(n * Kc));
    int64_t *excl = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * (Kc > L ? Kc : L)));
    int rc = 0;
    if (!knn_ids || !knn_d || !excl || !off || !cand) rc = -2;
    if (!rc) {
        for (int64_t u = 0; u < n; ++u) excl[u] = u;
        rc = or_knn(D, n, d, metric, D, n, excl, Kc, knn_ids, knn_d);
    }
    if (!rc) {
        memcpy(cand, knn_ids, sizeof(int32_t) * (size_t)(n * Kc));
        for (int64_t u = 0; u <= n; ++u) off[u] = u * Kc;
    }
    for (int it = 0; it < iters && !rc; ++it) {
        rc = refine(D, n, d, metric, off, cand, R, cos_alpha, alpha60, nbr, deg, 1, ep);
        if (!rc) rc = or_acquire(D, n, d, metric, nbr, deg, R, L, cand, NULL);
        if (!rc)
            for (int64_t u = 0; u <= n; ++u) off[u] = u * L;
    }
    if (!rc)
        rc = refine(D, n, d, metric, off, cand, R, cos_alpha_final, alpha_final60, nbr, deg,
                    connect_final, ep);
    free(knn_ids);
    free(knn_d);
    free(excl);
    free(off);
    free(cand);
    return rc ? rc : ep;
}

/* ---------------------------------------------------------------------- */
/* HNSW level draw (Algorithm 4, Algorithm 7): an                         */
/* exponentially decaying level l = floor(-ln(U) / ln(M)).  The uniform   */
/* U of point i comes from SplitMix64 (Steele, Lea and Flood, OOPSLA      */
/* 2014) seeded with seed XOR i: U = ((z >> 11) + 1) * 2^-53, in (0, 1].   */
/* ---------------------------------------------------------------------- */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

void or_levels(int64_t n, uint64_t seed, int M, int32_t *level)
{
    double lnM = log((double)M);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t z = splitmix64(seed ^ (uint64_t)i);
        double U = (double)((z >> 11) + 1) * (1.0 / 9007199254740992.0);
        level[i] = (int32_t)floor(-log(U) / lnM);
    }
}

/* ---------------------------------------------------------------------- */
/* kNN-graph refinement by 2-hop neighbours, the iteration of KGraph's      */
/* NN-descent as Exp. 12 describes it: starting from K neighbours per point */
/* (drawn at random; here an input), every iteration each point u computes  */
/* the distance to its 2-hop neighbours, and its new list is the K best by  */
/* (s, id) of its current neighbours and their neighbours, u excluded.      */
/* Lists are ordered by (s, id), -1 padded, repeated ids counted once.      */
/* cur [n][K] is read (the iteration's snapshot) and next [n][K] written.   */
/* ---------------------------------------------------------------------- */
static void descent_row(const float *D, int64_t n, int d, int metric, const int32_t *cur, int K,
                        int64_t u, int32_t *out_i, double *out_s, item_t *buf, int64_t *seen,
                        int64_t stamp)
{
    int m = 0;
    for (int a = 0; a < K; ++a) {
        const int32_t v = cur[u * K + a];
        if (v < 0) continue;
        for (int b = -1; b < K; ++b) {
            const int32_t w = b < 0 ? v : cur[(int64_t)v * K + b];
            if (w < 0 || w == u || seen[w] == stamp) continue;
            seen[w] = stamp;
            buf[m].s = or_dist(D + (size_t)u * d, D + (size_t)w * d, d, metric);
            buf[m].id = w;
            ++m;
        }
    }
    qsort(buf, (size_t)m, sizeof(item_t), item_cmp);
    for (int j = 0; j < K; ++j) {
        out_i[j] = j < m ? buf[j].id : -1;
        if (out_s) out_s[j] = j < m ? buf[j].s : INFINITY;
    }
}

int or_knn_descent(const float *D, int64_t n, int d, int metric, int K, int iters,
                   const int32_t *init, int32_t *ids, double *dist)
{
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * K));
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * K));
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return -2;
    }
    /* N_0(u): the initial ids themselves, sorted by (s, id) */
#pragma omp parallel
    {
        item_t *buf = (item_t *)malloc(sizeof(item_t) * (size_t)K);
#pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < n; ++u) {
            int m = 0;
            for (int a = 0; a < K; ++a) {
                const int32_t v = init[u * K + a];
                if (v < 0 || v >= n || v == u) continue;
                int dup = 0;
                for (int e = 0; e < m && !dup; ++e) dup = buf[e].id == v;
                if (dup) continue;
                buf[m].s = or_dist(D + (size_t)u * d, D + (size_t)v * d, d, metric);
                buf[m].id = v;
                ++m;
            }
            qsort(buf, (size_t)m, sizeof(item_t), item_cmp);
            for (int j = 0; j < K; ++j) cur[u * K + j] = j < m ? buf[j].id : -1;
        }
        free(buf);
    }
    for (int it = 0; it < iters; ++it) {
#pragma omp parallel
        {
            item_t *buf = (item_t *)malloc(sizeof(item_t) * (size_t)(K * (K + 1)));
            int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
            for (int64_t i = 0; i < n; ++i) seen[i] = -1;
#pragma omp for schedule(dynamic, 16)
            for (int64_t u = 0; u < n; ++u)
                descent_row(D, n, d, metric, cur, K, u, nxt + u * K, NULL, buf, seen, u);
            free(buf);
            free(seen);
        }
        int32_t *t = cur;
        cur = nxt;
        nxt = t;
    }
    for (int64_t u = 0; u < n; ++u)
        for (int j = 0; j < K; ++j) {
            const int32_t v = cur[u * K + j];
            ids[u * K + j] = v;
            dist[u * K + j] = v >= 0 ? or_dist(D + (size_t)u * d, D + (size_t)v * d, d, metric)
                                     : INFINITY;
        }
    free(cur);
    free(nxt);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
