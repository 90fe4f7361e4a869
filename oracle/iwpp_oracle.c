/*
 * CPU oracle for the irregular wavefront propagation pattern (IWPP) of
 * Teodoro et al., "Efficient Irregular Wavefront Propagation Algorithms on
 * Hybrid CPU-GPU Machines" (arXiv:1209.3314).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, sequential, obviously
 * correct reference that the CUDA path is checked against.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it; the
 * product library never links, includes or calls it, and it shares no code,
 * header or table with the CUDA sources.
 *
 * Contents
 *   oracle_fh_i32 / oracle_fh_u8  Fast hybrid grayscale reconstruction by
 *                                 dilation (Section 2.1, Algorithm 2).
 *   oracle_edt                    Wavefront-propagation distance transform
 *                                 (Section 2.2, Algorithm 3).
 *   oracle_edt_exact              Exact squared Euclidean distance transform
 *                                 by the separable method of Meijster,
 *                                 Roerdink and Hesselink (2000); used to count
 *                                 where Algorithm 3 departs from the exact
 *                                 distance (Section 2.2, Figure 3).
 *   oracle_gdt                    Shortest-path (geodesic) distance on a grid
 *                                 with obstacles, one of the IWPP uses named
 *                                 in Section 1, by Dijkstra's algorithm.
 *   oracle_skiz                   Influence zones and their skeleton (SKIZ)
 *                                 of labelled sources inside a mask, another
 *                                 IWPP use named in Section 1, by Dijkstra's
 *                                 algorithm and breadth-first searches per
 *                                 label along shortest-path edges.
 *   oracle_watershed              Marker-controlled watershed by flooding,
 *                                 another IWPP use named in Section 1:
 *                                 flooding levels by Dijkstra's algorithm on
 *                                 the highest-value path cost, plateau
 *                                 distances by breadth-first search, labels
 *                                 by breadth-first search per marker label.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - pixels outside the image do not exist (no padding, no wrap-around);
 *   - Algorithm 2's test "I(q) != J(q)" is taken as J(q) < I(q), identical
 *     once J <= I, which the raster pass establishes (it applies "and I(p)"
 *     to every pixel);
 *   - N+ (8-connected) = {(-1,-1), (-1,0), (-1,+1), (0,-1)} in (dy, dx) and
 *     N- is its point mirror; 4-connected: {(-1,0), (0,-1)} and mirror;
 *   - DIST is compared as exact integer squared distance (monotone in the
 *     Euclidean distance, no rounding); the virtual "inf" pixel is -1 and is
 *     farther than any real pixel;
 *   - distance-transform features are the pixels of the "background" class:
 *     value 0 by default (the paper's polarity), non-zero when
 *     feature_nonzero is set; an image without features yields nearest = -1
 *     and squared distance INT32_MAX.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ FIFO */

typedef struct {
    int64_t *buf;
    int64_t cap, head, tail; /* live items are buf[head..tail) */
} fifo_t;

static int fifo_init(fifo_t *f, int64_t cap) {
    if (cap < 16) cap = 16;
    f->buf = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    f->cap = cap;
    f->head = f->tail = 0;
    return f->buf ? 0 : -1;
}

static int fifo_push(fifo_t *f, int64_t v) {
    if (f->tail == f->cap) {
        int64_t live = f->tail - f->head;
        if (f->head > 0 && live <= f->cap / 2) {
            memmove(f->buf, f->buf + f->head, (size_t)live * sizeof(int64_t));
        } else {
            int64_t ncap = f->cap * 2;
            int64_t *nb = (int64_t *)malloc((size_t)ncap * sizeof(int64_t));
            if (!nb) return -1;
            memcpy(nb, f->buf + f->head, (size_t)live * sizeof(int64_t));
            free(f->buf);
            f->buf = nb;
            f->cap = ncap;
        }
        f->head = 0;
        f->tail = live;
    }
    f->buf[f->tail++] = v;
    return 0;
}

/* pop policy: 0 = FIFO (the paper's queue), 1 = LIFO, 2 = uniformly random
 * live item (xorshift64*), used only to probe order dependence. */
static int64_t fifo_pop(fifo_t *f, int policy, uint64_t *rng) {
    if (policy == 1) return f->buf[--f->tail];
    if (policy == 2) {
        uint64_t x = *rng;
        x ^= x >> 12; x ^= x << 25; x ^= x >> 27;
        *rng = x;
        int64_t live = f->tail - f->head;
        int64_t k = f->head + (int64_t)((x * 2685821657736338717ULL) % (uint64_t)live);
        int64_t v = f->buf[k];
        f->buf[k] = f->buf[f->head];
        f->head++;
        return v;
    }
    return f->buf[f->head++];
}

static void fifo_free(fifo_t *f) { free(f->buf); f->buf = NULL; }

/* ------------------------------------------------ neighbourhood offsets */

/* (dy, dx) pairs.  The first half of the 8-neighbourhood is N+ (reached
 * before p in raster order), the second half its mirror N-. */
static const int NB8[8][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1},
                              {1, 1},   {1, 0},  {1, -1}, {0, 1}};
static const int NB4[4][2] = {{-1, 0}, {0, -1}, {1, 0}, {0, 1}};

static inline int inside(int y, int x, int h, int w) {
    return y >= 0 && y < h && x >= 0 && x < w;
}

/* ----------------------------------------- reconstruction, Algorithm 2 */

/*
 * Fast hybrid reconstruction (Section 2.1, Algorithm 2) on int32 values.
 * I: mask (h*w, row-major), J: marker on entry, reconstruction on exit.
 * counters (may be NULL): [0] initial queue size after the anti-raster
 * pass, [1] total number of queue insertions.
 * Returns 0, or -1 on allocation failure / bad connectivity.
 */
int oracle_fh_i32(int h, int w, const int32_t *I, int32_t *J, int conn,
                  int64_t *counters) {
    if (conn != 4 && conn != 8) return -1;
    const int (*nb)[2] = conn == 8 ? NB8 : NB4;
    const int half = conn / 2; /* nb[0..half) = N+, nb[half..conn) = N- */
    fifo_t q;
    if (fifo_init(&q, (int64_t)h * w / 8 + 64)) return -1;

    /* Raster scan: J(p) <- max{J(q), q in N+(p) u {p}} and I(p). */
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int64_t p = (int64_t)y * w + x;
            int32_t m = J[p];
            for (int k = 0; k < half; k++) {
                int yy = y + nb[k][0], xx = x + nb[k][1];
                if (inside(yy, xx, h, w) && J[(int64_t)yy * w + xx] > m)
                    m = J[(int64_t)yy * w + xx];
            }
            J[p] = m < I[p] ? m : I[p];
        }

    /* Anti-raster scan with N-, then the queue test on N-. */
    for (int y = h - 1; y >= 0; y--)
        for (int x = w - 1; x >= 0; x--) {
            int64_t p = (int64_t)y * w + x;
            int32_t m = J[p];
            for (int k = half; k < conn; k++) {
                int yy = y + nb[k][0], xx = x + nb[k][1];
                if (inside(yy, xx, h, w) && J[(int64_t)yy * w + xx] > m)
                    m = J[(int64_t)yy * w + xx];
            }
            J[p] = m < I[p] ? m : I[p];
            for (int k = half; k < conn; k++) {
                int yy = y + nb[k][0], xx = x + nb[k][1];
                if (!inside(yy, xx, h, w)) continue;
                int64_t qq = (int64_t)yy * w + xx;
                if (J[qq] < J[p] && J[qq] < I[qq]) {
                    if (fifo_push(&q, p)) { fifo_free(&q); return -1; }
                    break;
                }
            }
        }
    int64_t initial = q.tail - q.head, pushes = initial;

    /* Wavefront propagation with a FIFO. */
    uint64_t dummy = 0;
    while (q.tail > q.head) {
        int64_t p = fifo_pop(&q, 0, &dummy);
        int y = (int)(p / w), x = (int)(p % w);
        for (int k = 0; k < conn; k++) {
            int yy = y + nb[k][0], xx = x + nb[k][1];
            if (!inside(yy, xx, h, w)) continue;
            int64_t qq = (int64_t)yy * w + xx;
            if (J[qq] < J[p] && J[qq] < I[qq]) {
                J[qq] = J[p] < I[qq] ? J[p] : I[qq];
                if (fifo_push(&q, qq)) { fifo_free(&q); return -1; }
                pushes++;
            }
        }
    }
    fifo_free(&q);
    if (counters) { counters[0] = initial; counters[1] = pushes; }
    return 0;
}

/* uint8 images: widened to int32, reconstructed, narrowed (values stay in
 * [0, 255] because every result lies between marker-and-mask and mask). */
int oracle_fh_u8(int h, int w, const uint8_t *I, uint8_t *J, int conn,
                 int64_t *counters) {
    int64_t n = (int64_t)h * w;
    int32_t *I32 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *J32 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!I32 || !J32) { free(I32); free(J32); return -1; }
    for (int64_t i = 0; i < n; i++) { I32[i] = I[i]; J32[i] = J[i]; }
    int rc = oracle_fh_i32(h, w, I32, J32, conn, counters);
    if (rc == 0)
        for (int64_t i = 0; i < n; i++) J[i] = (uint8_t)J32[i];
    free(I32); free(J32);
    return rc;
}

/* -------------------------------------- distance transform, Algorithm 3 */

static inline int64_t sqd(int64_t a, int64_t b, int w) {
    /* squared distance between linear pixel indices a and b (b >= 0) */
    int64_t dy = a / w - b / w, dx = a % w - b % w;
    return dy * dy + dx * dx;
}

/*
 * Wavefront-propagation distance transform (Section 2.2, Algorithm 3),
 * 8-connected.  bin: h*w uint8; features are bin==0 (feature_nonzero=0) or
 * bin!=0 (feature_nonzero=1).  Outputs: nearest[p] = linear index of the
 * feature assigned to p (VR), sqdist[p] = squared distance to it.
 * policy: 0 FIFO (the algorithm as published), 1 LIFO, 2 random (seeded by
 * seed) -- the last two only probe how the result depends on pop order.
 * counters (may be NULL): [0] initial queue size, [1] total insertions.
 */
int oracle_edt_policy(int h, int w, const uint8_t *bin, int feature_nonzero,
                      int32_t *nearest, int32_t *sqdist, int64_t *counters,
                      int policy, uint64_t seed) {
    int64_t n = (int64_t)h * w;
    int64_t *VR = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!VR) return -1;
    fifo_t q;
    if (fifo_init(&q, n / 8 + 64)) { free(VR); return -1; }
#define IS_FEATURE(i) (feature_nonzero ? bin[i] != 0 : bin[i] == 0)

    /* Initialization: VR(p) = p for features, inf (-1) otherwise; queue the
     * features that have a non-feature 8-neighbour, in raster order. */
    for (int64_t p = 0; p < n; p++) VR[p] = IS_FEATURE(p) ? p : -1;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int64_t p = (int64_t)y * w + x;
            if (!IS_FEATURE(p)) continue;
            for (int k = 0; k < 8; k++) {
                int yy = y + NB8[k][0], xx = x + NB8[k][1];
                if (inside(yy, xx, h, w) && !IS_FEATURE((int64_t)yy * w + xx)) {
                    if (fifo_push(&q, p)) { fifo_free(&q); free(VR); return -1; }
                    break;
                }
            }
        }
    int64_t initial = q.tail - q.head, pushes = initial;

    /* Propagation: q takes VR(p) when that feature is strictly closer. */
    uint64_t rng = seed * 0x9E3779B97F4A7C15ULL + 1;
    while (q.tail > q.head) {
        int64_t p = fifo_pop(&q, policy, &rng);
        int y = (int)(p / w), x = (int)(p % w);
        int64_t f = VR[p];
        for (int k = 0; k < 8; k++) {
            int yy = y + NB8[k][0], xx = x + NB8[k][1];
            if (!inside(yy, xx, h, w)) continue;
            int64_t qq = (int64_t)yy * w + xx;
            int64_t dnew = sqd(qq, f, w);
            if (VR[qq] < 0 || dnew < sqd(qq, VR[qq], w)) {
                VR[qq] = f;
                if (fifo_push(&q, qq)) { fifo_free(&q); free(VR); return -1; }
                pushes++;
            }
        }
    }
#undef IS_FEATURE
    /* Distance map from the Voronoi assignment. */
    for (int64_t p = 0; p < n; p++) {
        if (VR[p] < 0) { nearest[p] = -1; sqdist[p] = INT32_MAX; }
        else { nearest[p] = (int32_t)VR[p]; sqdist[p] = (int32_t)sqd(p, VR[p], w); }
    }
    fifo_free(&q);
    free(VR);
    if (counters) { counters[0] = initial; counters[1] = pushes; }
    return 0;
}

int oracle_edt(int h, int w, const uint8_t *bin, int feature_nonzero,
               int32_t *nearest, int32_t *sqdist, int64_t *counters) {
    return oracle_edt_policy(h, w, bin, feature_nonzero, nearest, sqdist,
                             counters, 0, 0);
}

/* ------------------------------------------------ exact squared EDT */

/*
 * Exact squared Euclidean distance to the nearest feature, by the two-phase
 * separable method of Meijster, Roerdink & Hesselink (2000):
 *   phase 1, per column: g(y) = distance to the nearest feature in that
 *            column (downward then upward scan);
 *   phase 2, per row: the lower envelope of the parabolas
 *            f_u(x) = (x - u)^2 + g(u)^2, found with a stack of parabola
 *            indices and their separation points, then read off left to right.
 * out: int32 squared distance, INT32_MAX where no feature exists.
 */
int oracle_edt_exact(int h, int w, const uint8_t *bin, int feature_nonzero,
                     int32_t *out) {
    const int64_t INF = (int64_t)h + w + 2; /* exceeds any real distance */
    int64_t *g = (int64_t *)malloc((size_t)h * w * sizeof(int64_t));
    int64_t *s = (int64_t *)malloc((size_t)w * sizeof(int64_t));
    int64_t *t = (int64_t *)malloc((size_t)w * sizeof(int64_t));
    if (!g || !s || !t) { free(g); free(s); free(t); return -1; }
#define FEAT(y, x) (feature_nonzero ? bin[(int64_t)(y) * w + (x)] != 0 \
                                    : bin[(int64_t)(y) * w + (x)] == 0)
    for (int x = 0; x < w; x++) {
        g[x] = FEAT(0, x) ? 0 : INF;
        for (int y = 1; y < h; y++)
            g[(int64_t)y * w + x] = FEAT(y, x) ? 0 : 1 + g[(int64_t)(y - 1) * w + x];
        for (int y = h - 2; y >= 0; y--) {
            int64_t below = g[(int64_t)(y + 1) * w + x];
            if (below < g[(int64_t)y * w + x]) g[(int64_t)y * w + x] = 1 + below;
        }
    }
#undef FEAT
    for (int y = 0; y < h; y++) {
        const int64_t *gy = g + (int64_t)y * w;
        int k = 0;
        s[0] = 0; t[0] = 0;
        for (int u = 1; u < w; u++) {
            /* pop parabolas that the new one beats at their start point */
            while (k >= 0) {
                int64_t a = t[k] - s[k], b = t[k] - u;
                if (a * a + gy[s[k]] * gy[s[k]] <= b * b + gy[u] * gy[u]) break;
                k--;
            }
            if (k < 0) { k = 0; s[0] = u; t[0] = 0; continue; }
            /* first x where parabola u is no worse than parabola s[k] */
            int64_t i = s[k];
            int64_t num = (int64_t)u * u - i * i + gy[u] * gy[u] - gy[i] * gy[i];
            int64_t sep = num / (2 * (u - i));
            int64_t start = sep + 1;
            if (start < w) { k++; s[k] = u; t[k] = start; }
        }
        for (int x = w - 1; x >= 0; x--) {
            int64_t dx = x - s[k], gv = gy[s[k]];
            int64_t d = gv >= INF ? -1 : dx * dx + gv * gv;
            out[(int64_t)y * w + x] = (d < 0 || d > INT32_MAX) ? INT32_MAX : (int32_t)d;
            if (x == t[k]) k--;
        }
    }
    free(g); free(s); free(t);
    return 0;
}

/* ------------------------------------ shortest paths on a grid (Section 1) */

/*
 * Geodesic distance from source pixels through free pixels, avoiding
 * obstacles: the shortest-path computation on a grid with obstacles that
 * Section 1 names as an instance of the IWPP.  The grid and the step costs
 * are this build's choice (the paper gives none):
 *   free(p)   = mask[p] != 0 (0 = obstacle);
 *   sources   = free pixels with seed[p] != 0;
 *   moves     = to any free 8-neighbour, cost 5 (horizontal or vertical)
 *               or 7 (diagonal) -- the 5-7 chamfer weights;
 *   dist[p]   = least total cost of a path from any source to p;
 *               INT32_MAX for obstacles and unreachable pixels.
 * Computed by Dijkstra's algorithm with a binary heap (lazy deletion: a
 * popped entry whose key exceeds the current distance is skipped).
 * stats (optional): [0] heap pops, [1] relaxations that improved a pixel.
 */
typedef struct { int64_t key; int64_t idx; } heap_item;

static void heap_push(heap_item *hp, int64_t *n, int64_t key, int64_t idx) {
    int64_t i = (*n)++;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (hp[parent].key <= key) break;
        hp[i] = hp[parent];
        i = parent;
    }
    hp[i].key = key;
    hp[i].idx = idx;
}

static heap_item heap_pop(heap_item *hp, int64_t *n) {
    heap_item top = hp[0], last = hp[--(*n)];
    int64_t i = 0;
    while (1) {
        int64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && hp[c + 1].key < hp[c].key) c++;
        if (last.key <= hp[c].key) break;
        hp[i] = hp[c];
        i = c;
    }
    if (*n > 0) hp[i] = last;
    return top;
}

int oracle_gdt(int h, int w, const uint8_t *mask, const uint8_t *seed, int32_t *dist,
               int64_t *stats) {
    const int64_t n = (int64_t)h * w;
    /* every improvement pushes one entry: at most 8 per pixel plus sources */
    heap_item *hp = (heap_item *)malloc((size_t)(9 * n + 1) * sizeof(heap_item));
    if (!hp) return -1;
    int64_t hn = 0, pops = 0, relax = 0;
    for (int64_t i = 0; i < n; i++) {
        dist[i] = INT32_MAX;
        if (mask[i] && seed[i]) {
            dist[i] = 0;
            heap_push(hp, &hn, 0, i);
        }
    }
    while (hn > 0) {
        heap_item it = heap_pop(hp, &hn);
        pops++;
        if (it.key > dist[it.idx]) continue; /* stale entry */
        const int y = (int)(it.idx / w), x = (int)(it.idx % w);
        for (int k = 0; k < 8; k++) {
            const int qy = y + NB8[k][0], qx = x + NB8[k][1];
            if (!inside(qy, qx, h, w)) continue;
            const int64_t q = (int64_t)qy * w + qx;
            if (!mask[q]) continue;
            const int64_t cost = (NB8[k][0] != 0 && NB8[k][1] != 0) ? 7 : 5;
            const int64_t nd = it.key + cost;
            if (nd < dist[q]) {
                dist[q] = (int32_t)nd;
                heap_push(hp, &hn, nd, q);
                relax++;
            }
        }
    }
    free(hp);
    if (stats) { stats[0] = pops; stats[1] = relax; }
    return 0;
}


/* ------------------------------------- watershed from markers (Section 1) */

/*
 * Marker-controlled watershed by flooding, named in Section 1 as an IWPP
 * algorithm.  The paper defines none; the definition taken here is the
 * image foresting transform with the highest-value path cost (Falcao,
 * Stolfi and Lotufo, 2004) and the lexicographic plateau cost of Lotufo and
 * Falcao (2000), with ties between basins settled by the least label:
 *   f         relief, int32 (uint8 reliefs are widened by the caller);
 *   markers   int32, 0 = no marker;
 *   a path's cost is the highest relief value on it (both ends included);
 *   level[p]  least cost of an 8-connected path from a marker pixel to p
 *             (the flooding level; f[p] at a marker pixel);
 *   pdist[p]  plateau distance: 0 at marker pixels and at pixels with a
 *             neighbour of lower level (the entry of p's level region),
 *             else 1 + the least pdist over neighbours of equal level;
 *   optimal edge p -> q (q a neighbour of p, q not a marker):
 *             level[p] < level[q] and pdist[q] = 0, or
 *             level[p] = level[q] and pdist[p] + 1 = pdist[q];
 *   label[q]  the least marker value among the marker pixels from which q
 *             is reached along optimal edges (a marker pixel keeps its own).
 * Optimal edges raise (level, pdist) strictly, so every label is settled by
 * the labels below it and the result does not depend on any visiting order.
 * Without markers nothing is reached: label 0, level and pdist INT32_MAX.
 *
 * Steps: (1) Dijkstra's algorithm on the highest-value cost from all marker
 * pixels (binary heap, lazy deletion); (2) breadth-first search from every
 * entry pixel at once across neighbours of equal level; (3) for each marker
 * value in increasing order, a breadth-first search along optimal edges
 * from its marker pixels that labels the pixels not labelled yet (a pixel
 * reached earlier carries a smaller label, and what lies behind it is then
 * reached with that smaller label as well).
 * stats (optional): [0] heap pops, [1] level improvements, [2] plateau
 * pushes, [3] label pushes.  Returns 0, or -1 on allocation failure.
 */
static int cmp_pair(const void *a, const void *b) {
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return x[1] < y[1] ? -1 : (x[1] > y[1] ? 1 : 0);
}

int oracle_watershed(int h, int w, const int32_t *f, const int32_t *markers,
                     int32_t *label, int32_t *level, int32_t *pdist,
                     int64_t *stats) {
    const int64_t n = (int64_t)h * w;
    int64_t nm = 0;
    for (int64_t i = 0; i < n; i++) nm += markers[i] != 0;
    heap_item *hp = (heap_item *)malloc((size_t)(9 * n + 1) * sizeof(heap_item));
    int64_t *lv = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *pairs = (int64_t *)malloc((size_t)(2 * nm + 2) * sizeof(int64_t));
    uint8_t *done = (uint8_t *)calloc((size_t)n + 1, 1);
    fifo_t q;
    if (!hp || !lv || !pairs || !done || fifo_init(&q, n + 1) != 0) {
        free(hp); free(lv); free(pairs); free(done);
        return -1;
    }
    const int64_t INF = INT64_MAX;
    int64_t hn = 0, pops = 0, improv = 0, ppush = 0, lpush = 0;

    /* (1) flooding levels */
    for (int64_t i = 0; i < n; i++) {
        lv[i] = INF;
        if (markers[i]) {
            lv[i] = f[i];
            heap_push(hp, &hn, lv[i], i);
        }
    }
    while (hn > 0) {
        heap_item it = heap_pop(hp, &hn);
        pops++;
        if (it.key > lv[it.idx]) continue; /* stale entry */
        const int y = (int)(it.idx / w), x = (int)(it.idx % w);
        for (int k = 0; k < 8; k++) {
            const int qy = y + NB8[k][0], qx = x + NB8[k][1];
            if (!inside(qy, qx, h, w)) continue;
            const int64_t qq = (int64_t)qy * w + qx;
            const int64_t c = it.key > f[qq] ? it.key : f[qq];
            if (c < lv[qq]) {
                lv[qq] = c;
                heap_push(hp, &hn, c, qq);
                improv++;
            }
        }
    }

    /* (2) plateau distances: entry pixels first, then breadth-first across
     * equal levels */
    for (int64_t i = 0; i < n; i++) {
        pdist[i] = INT32_MAX;
        if (lv[i] == INF) continue;
        int entry = markers[i] != 0;
        const int y = (int)(i / w), x = (int)(i % w);
        for (int k = 0; k < 8 && !entry; k++) {
            const int qy = y + NB8[k][0], qx = x + NB8[k][1];
            if (inside(qy, qx, h, w) && lv[(int64_t)qy * w + qx] < lv[i]) entry = 1;
        }
        if (entry) {
            pdist[i] = 0;
            fifo_push(&q, i);
            ppush++;
        }
    }
    while (q.head < q.tail) {
        const int64_t p = fifo_pop(&q, 0, NULL);
        const int y = (int)(p / w), x = (int)(p % w);
        for (int k = 0; k < 8; k++) {
            const int qy = y + NB8[k][0], qx = x + NB8[k][1];
            if (!inside(qy, qx, h, w)) continue;
            const int64_t qq = (int64_t)qy * w + qx;
            if (lv[qq] == lv[p] && pdist[qq] == INT32_MAX) {
                pdist[qq] = pdist[p] + 1;
                fifo_push(&q, qq);
                ppush++;
            }
        }
    }

    /* (3) labels, one marker value at a time in increasing order */
    int64_t np = 0;
    for (int64_t i = 0; i < n; i++) {
        label[i] = markers[i];
        if (markers[i]) {
            pairs[2 * np] = markers[i];
            pairs[2 * np + 1] = i;
            np++;
            done[i] = 1;
        }
    }
    qsort(pairs, (size_t)np, 2 * sizeof(int64_t), cmp_pair);
    for (int64_t a = 0; a < np;) {
        int64_t b = a;
        q.head = q.tail = 0;
        while (b < np && pairs[2 * b] == pairs[2 * a]) {
            fifo_push(&q, pairs[2 * b + 1]);
            b++;
        }
        const int32_t L = (int32_t)pairs[2 * a];
        while (q.head < q.tail) {
            const int64_t p = fifo_pop(&q, 0, NULL);
            const int y = (int)(p / w), x = (int)(p % w);
            for (int k = 0; k < 8; k++) {
                const int qy = y + NB8[k][0], qx = x + NB8[k][1];
                if (!inside(qy, qx, h, w)) continue;
                const int64_t qq = (int64_t)qy * w + qx;
                if (done[qq]) continue; /* a marker, or labelled by a smaller value */
                const int rise = lv[p] < lv[qq] && pdist[qq] == 0;
                const int flat = lv[p] == lv[qq] && (int64_t)pdist[p] + 1 == pdist[qq];
                if (rise || flat) {
                    label[qq] = L;
                    done[qq] = 1;
                    fifo_push(&q, qq);
                    lpush++;
                }
            }
        }
        a = b;
    }
    for (int64_t i = 0; i < n; i++) level[i] = lv[i] == INF ? INT32_MAX : (int32_t)lv[i];
    fifo_free(&q);
    free(hp); free(lv); free(pairs); free(done);
    if (stats) { stats[0] = pops; stats[1] = improv; stats[2] = ppush; stats[3] = lpush; }
    return 0;
}

/* ------------------------- influence zones and SKIZ (Section 1) */

/*
 * Influence zones of labelled sources inside a mask and their skeleton
 * (SKIZ), named in Section 1 among the IWPP algorithms.  The paper defines
 * neither; the definition taken here is the geodesic SKIZ (Lantuejoul,
 * 1980) with the grid metric of oracle_gdt:
 *   free(p)   = mask[p] != 0; sources: free pixels with labels[p] != 0;
 *   dist[p]   = least cost of a path through free pixels from any source
 *               (8 moves, cost 5 straight / 7 diagonal), as oracle_gdt;
 *   a label L reaches p when the least cost from the sources labelled L
 *               equals dist[p];
 *   zones[p]  = the least label that reaches p (0 at obstacles and
 *               unreachable pixels);
 *   skiz[p]   = 1 when two or more labels reach p, else 0.
 * A label reaches p exactly when p lies on a shortest path from one of its
 * sources, i.e. along edges q -> p with dist[q] + cost = dist[p] (every
 * prefix of a shortest path is shortest).  So: Dijkstra's algorithm for
 * dist, then for each label value in increasing order a breadth-first
 * search along such edges from its sources that marks the pixels not
 * reached yet (the least label), and the same in decreasing order (the
 * greatest); two labels reach p exactly when the two differ.
 * Returns 0, or -1 on allocation failure.
 */
static void skiz_sweep(int h, int w, const uint8_t *mask, const int32_t *dist,
                       const int64_t *pairs, int64_t np, int descending,
                       int32_t *out, uint8_t *done, fifo_t *q) {
    const int64_t n = (int64_t)h * w;
    memset(done, 0, (size_t)n);
    for (int64_t i = 0; i < np; i++) done[pairs[2 * i + 1]] = 1;
    for (int64_t g = 0; g < np;) {
        const int64_t a = descending ? np - 1 - g : g;
        int64_t cnt = 0;
        q->head = q->tail = 0;
        while (g + cnt < np) {
            const int64_t b = descending ? np - 1 - (g + cnt) : g + cnt;
            if (pairs[2 * b] != pairs[2 * a]) break;
            fifo_push(q, pairs[2 * b + 1]);
            cnt++;
        }
        const int32_t L = (int32_t)pairs[2 * a];
        while (q->head < q->tail) {
            const int64_t p = fifo_pop(q, 0, NULL);
            const int y = (int)(p / w), x = (int)(p % w);
            for (int k = 0; k < 8; k++) {
                const int qy = y + NB8[k][0], qx = x + NB8[k][1];
                if (!inside(qy, qx, h, w)) continue;
                const int64_t qq = (int64_t)qy * w + qx;
                if (done[qq] || !mask[qq] || dist[qq] == INT32_MAX) continue;
                const int64_t cost = (NB8[k][0] != 0 && NB8[k][1] != 0) ? 7 : 5;
                if ((int64_t)dist[p] + cost == dist[qq]) {
                    out[qq] = L;
                    done[qq] = 1;
                    fifo_push(q, qq);
                }
            }
        }
        g += cnt;
    }
}

int oracle_skiz(int h, int w, const uint8_t *mask, const int32_t *labels,
                int32_t *zones, uint8_t *skiz, int32_t *dist) {
    const int64_t n = (int64_t)h * w;
    uint8_t *seed = (uint8_t *)malloc((size_t)n + 1);
    int32_t *zmax = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    uint8_t *done = (uint8_t *)malloc((size_t)n + 1);
    int64_t np = 0;
    for (int64_t i = 0; i < n; i++) np += mask[i] && labels[i];
    int64_t *pairs = (int64_t *)malloc((size_t)(2 * np + 2) * sizeof(int64_t));
    fifo_t q;
    if (!seed || !zmax || !done || !pairs || fifo_init(&q, n + 1) != 0) {
        free(seed); free(zmax); free(done); free(pairs);
        return -1;
    }
    np = 0;
    for (int64_t i = 0; i < n; i++) {
        seed[i] = labels[i] != 0;
        zones[i] = zmax[i] = 0;
        if (mask[i] && labels[i]) {
            zones[i] = zmax[i] = labels[i];
            pairs[2 * np] = labels[i];
            pairs[2 * np + 1] = i;
            np++;
        }
    }
    int rc = oracle_gdt(h, w, mask, seed, dist, NULL);
    if (rc == 0) {
        qsort(pairs, (size_t)np, 2 * sizeof(int64_t), cmp_pair);
        skiz_sweep(h, w, mask, dist, pairs, np, 0, zones, done, &q);
        skiz_sweep(h, w, mask, dist, pairs, np, 1, zmax, done, &q);
        for (int64_t i = 0; i < n; i++) skiz[i] = zones[i] != zmax[i];
    }
    fifo_free(&q);
    free(seed); free(zmax); free(done); free(pairs);
    return rc;
}
