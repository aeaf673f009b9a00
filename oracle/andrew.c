/*
 * oracle/andrew.c -- CPU oracle for the convex hull.  TEST INFRASTRUCTURE ONLY:
 * nothing in the product path links, loads or calls this file; only the tests,
 * the smoke check and the benchmark's CPU-baseline leg do.  It shares no code,
 * header or constant with the CUDA library.
 *
 * What it computes (the plain definition the GPU path must reach exactly):
 * the convex hull of ALL n input points -- the problem of Alg. 1 (input
 * P[1..n], output CH[1..h] in counter-clockwise order) -- as the list of the
 * indices of the strictly convex hull vertices, counter-clockwise, starting at
 * the lexicographically smallest (x, then y) vertex.  Points on a hull edge
 * that are not corners are excluded.  A vertex whose coordinates occur several
 * times is represented by the lowest index carrying them.
 *
 * Algorithm: Andrew's monotone chain (1979; Table I lists it among the
 * O(n log n) hull algorithms):
 *   1. check every coordinate is an integer in [0, 2^24); convert to int64;
 *   2. sort the points by (x, y, index);
 *   3. keep the first point of every run of equal (x, y);
 *   4. with at most two distinct points, output them in that order;
 *   5. lower chain: scan ascending, popping while cross(o, a, b) <= 0;
 *   6. upper chain: scan descending with the same rule;
 *   7. concatenate the chains without their repeated end points.
 * cross(o, a, b) = (a.x - o.x)(b.y - o.y) - (a.y - o.y)(b.x - o.x) is exact in
 * int64: operands are below 2^24, products below 2^48.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_OK 0
#define ORACLE_ERANGE (-2)
#define ORACLE_ENOMEM (-3)

typedef struct {
    int64_t x, y;
    int64_t idx;
} opoint;

static int cmp_xy_idx(const void* pa, const void* pb) {
    const opoint* a = (const opoint*)pa;
    const opoint* b = (const opoint*)pb;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static int64_t cross3(const opoint* o, const opoint* a, const opoint* b) {
    return (a->x - o->x) * (b->y - o->y) - (a->y - o->y) * (b->x - o->x);
}

/* 1 if v is an integer-valued float in [0, 2^24); NaN and infinities fail. */
static int coord_ok(float v) {
    return v >= 0.0f && v < 16777216.0f && v == floorf(v);
}

/* Returns ORACLE_OK when every coordinate is in the input domain, else ORACLE_ERANGE. */
int oracle_check(const float* pts, int64_t n) {
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!coord_ok(pts[i])) return ORACLE_ERANGE;
    return ORACLE_OK;
}

/*
 * Hull of pts[0..n) (x, y interleaved).  Writes h indices to out_idx (capacity
 * n) and returns h, or a negative status.
 */
int64_t oracle_hull(const float* pts, int64_t n, int32_t* out_idx) {
    if (n < 0) return ORACLE_ERANGE;
    if (oracle_check(pts, n) != ORACLE_OK) return ORACLE_ERANGE;
    if (n == 0) return 0;

    opoint* p = (opoint*)malloc((size_t)n * sizeof(opoint));
    if (!p) return ORACLE_ENOMEM;
    for (int64_t i = 0; i < n; ++i) {
        p[i].x = (int64_t)pts[2 * i];
        p[i].y = (int64_t)pts[2 * i + 1];
        p[i].idx = i;
    }
    qsort(p, (size_t)n, sizeof(opoint), cmp_xy_idx);

    /* Step 3: the first of each equal-(x, y) run has the lowest index. */
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (m > 0 && p[m - 1].x == p[i].x && p[m - 1].y == p[i].y) continue;
        p[m++] = p[i];
    }

    if (m <= 2) {
        for (int64_t i = 0; i < m; ++i) out_idx[i] = (int32_t)p[i].idx;
        free(p);
        return m;
    }

    opoint* h = (opoint*)malloc((size_t)(2 * m) * sizeof(opoint));
    if (!h) {
        free(p);
        return ORACLE_ENOMEM;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {                     /* lower chain */
        while (k >= 2 && cross3(&h[k - 2], &h[k - 1], &p[i]) <= 0) --k;
        h[k++] = p[i];
    }
    const int64_t lower_len = k + 1;
    for (int64_t i = m - 2; i >= 0; --i) {                /* upper chain */
        while (k >= lower_len && cross3(&h[k - 2], &h[k - 1], &p[i]) <= 0) --k;
        h[k++] = p[i];
    }
    --k; /* the last point repeats the first */
    for (int64_t i = 0; i < k; ++i) out_idx[i] = (int32_t)h[i].idx;
    free(h);
    free(p);
    return k;
}
