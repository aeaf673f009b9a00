/*
 * oracle/heaphull_cpu.c -- the paper's heaphull on the host's cores: the CPU
 * comparator that the benchmark times beside the GPU path.  TEST AND
 * MEASUREMENT INFRASTRUCTURE ONLY: the CUDA library never links, loads or
 * calls it, and it shares no code with it.  It is not the oracle's definition
 * (andrew.c is); its results are checked against andrew.c by the tests.
 *
 * Steps, on T threads (POSIX threads, contiguous chunks of the input):
 *   1. findExtremes (Alg. 2; Sec. 3): per chunk the 8 directional extremes,
 *      argmin / argmax of x, y, x + y and x - y with the lowest index on
 *      ties, then the minimum / maximum over the chunks.
 *   2. The filter of Alg. 1 / 2: a point strictly inside the octagon of the
 *      extremes (strictly left of every edge of non-zero length, octagon of
 *      non-zero area) is interior to the hull and is dropped; every other
 *      point survives (a superset of the four queues of Alg. 1).
 *   3. "CH <- union of hull(Q_i)": the survivors hold every hull vertex and
 *      every repetition of its coordinates, so Andrew's monotone chain
 *      (Table I) over them gives the hull of all points.  They are ordered
 *      by (x, y, index) with a parallel sort (per-chunk qsort, then pairwise
 *      merges in parallel rounds); the chains themselves are sequential.
 * Output convention as andrew.c: strictly convex vertices, counter-clockwise
 * from the lexicographically smallest, the lowest index per coordinate.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HH_OK 0
#define HH_ERANGE (-2)
#define HH_ENOMEM (-3)
#define HH_MAX_THREADS 256

typedef struct {
    int64_t x, y, idx;
} hpt;

/* direction order W, SW, S, SE, E, NE, N, NW (counter-clockwise around the
 * hull); key d is minimised for W, SW, S, NW and maximised for SE, E, NE, N */
static int64_t dir_key(int d, int64_t x, int64_t y) {
    switch (d) {
        case 0: case 4: return x;
        case 2: case 6: return y;
        case 1: case 5: return x + y;
        default: return x - y;
    }
}
static int dir_max(int d) { return d >= 3 && d <= 6; }

static int coord_ok(float v) { return v >= 0.0f && v < 16777216.0f && v == floorf(v); }

static int64_t cross3(int64_t ox, int64_t oy, int64_t ax, int64_t ay, int64_t bx, int64_t by) {
    return (ax - ox) * (by - oy) - (ay - oy) * (bx - ox);
}

static int cmp_pt(const void* pa, const void* pb) {
    const hpt* a = (const hpt*)pa;
    const hpt* b = (const hpt*)pb;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* ---------------------------------------------------------------------- */
typedef struct {
    const float* pts;
    int64_t lo, hi;
    int bad;
    int64_t key[8], arg[8];   /* step 1 */
    const int64_t* ox;        /* step 2: octagon vertices (8), NULL = keep all */
    const int64_t* oy;
    hpt* surv;                /* step 2: this chunk's survivors */
    int64_t nsurv;
    hpt* a;                   /* step 3: sort / merge ranges */
    hpt* b;
    int64_t m0, m1, m2;
} job;

static void* run_extremes(void* arg) {
    job* j = (job*)arg;
    j->bad = 0;
    for (int d = 0; d < 8; ++d) {
        j->key[d] = dir_max(d) ? INT64_MIN : INT64_MAX;
        j->arg[d] = -1;
    }
    for (int64_t i = j->lo; i < j->hi; ++i) {
        const float fx = j->pts[2 * i], fy = j->pts[2 * i + 1];
        if (!coord_ok(fx) || !coord_ok(fy)) {
            j->bad = 1;
            return NULL;
        }
        const int64_t x = (int64_t)fx, y = (int64_t)fy;
        for (int d = 0; d < 8; ++d) {   /* strict improvement keeps the lowest index */
            const int64_t k = dir_key(d, x, y);
            if (dir_max(d) ? k > j->key[d] : k < j->key[d]) {
                j->key[d] = k;
                j->arg[d] = i;
            }
        }
    }
    return NULL;
}

static void* run_filter(void* arg) {
    job* j = (job*)arg;
    int64_t m = 0;
    for (int64_t i = j->lo; i < j->hi; ++i) {
        const int64_t x = (int64_t)j->pts[2 * i], y = (int64_t)j->pts[2 * i + 1];
        int inside = j->ox != NULL;
        for (int e = 0; e < 8 && inside; ++e) {
            const int f = (e + 1) & 7;
            if (j->ox[e] == j->ox[f] && j->oy[e] == j->oy[f]) continue;   /* zero-length edge */
            if (cross3(j->ox[e], j->oy[e], j->ox[f], j->oy[f], x, y) <= 0) inside = 0;
        }
        if (inside) continue;
        j->surv[m].x = x;
        j->surv[m].y = y;
        j->surv[m].idx = i;
        ++m;
    }
    j->nsurv = m;
    return NULL;
}

static void* run_sort(void* arg) {
    job* j = (job*)arg;
    qsort(j->a + j->m0, (size_t)(j->m1 - j->m0), sizeof(hpt), cmp_pt);
    return NULL;
}

/* merges a[m0, m1) and a[m1, m2) into b[m0, m2) */
static void* run_merge(void* arg) {
    job* j = (job*)arg;
    int64_t p = j->m0, q = j->m1, o = j->m0;
    while (p < j->m1 && q < j->m2) j->b[o++] = cmp_pt(&j->a[q], &j->a[p]) < 0 ? j->a[q++] : j->a[p++];
    while (p < j->m1) j->b[o++] = j->a[p++];
    while (q < j->m2) j->b[o++] = j->a[q++];
    return NULL;
}

static void run_all(void* (*fn)(void*), job* jobs, int t) {
    pthread_t th[HH_MAX_THREADS];
    int started[HH_MAX_THREADS];
    for (int i = 1; i < t; ++i) started[i] = pthread_create(&th[i], NULL, fn, &jobs[i]) == 0;
    fn(&jobs[0]);
    for (int i = 1; i < t; ++i) {
        if (started[i]) pthread_join(th[i], NULL);
        else fn(&jobs[i]);   /* no thread to spare: run it here */
    }
}

/*
 * Hull of pts[0..n) (x, y interleaved) on `threads` threads (<= 0: 1).
 * Writes h indices to out_idx (capacity n) and returns h, or a negative
 * status (HH_ERANGE for a coordinate outside the integers of [0, 2^24)).
 */
int64_t cpu_heaphull(const float* pts, int64_t n, int32_t* out_idx, int threads) {
    if (n < 0) return HH_ERANGE;
    if (n == 0) return 0;
    int t = threads < 1 ? 1 : (threads > HH_MAX_THREADS ? HH_MAX_THREADS : threads);
    if ((int64_t)t > n) t = (int)n;
    job* jobs = (job*)calloc((size_t)t, sizeof(job));
    hpt* surv = (hpt*)malloc((size_t)n * sizeof(hpt));
    hpt* tmp = NULL;
    int64_t result = HH_ENOMEM;
    if (!jobs || !surv) goto done;
    for (int i = 0; i < t; ++i) {
        jobs[i].pts = pts;
        jobs[i].lo = n * i / t;
        jobs[i].hi = n * (i + 1) / t;
    }
    /* 1. extremes */
    run_all(run_extremes, jobs, t);
    int64_t key[8], ext[8];
    for (int d = 0; d < 8; ++d) {
        key[d] = jobs[0].key[d];
        ext[d] = jobs[0].arg[d];
    }
    for (int i = 0; i < t; ++i) {
        if (jobs[i].bad) {
            result = HH_ERANGE;
            goto done;
        }
        for (int d = 0; d < 8; ++d) {   /* chunks in index order: strict improvement */
            if (dir_max(d) ? jobs[i].key[d] > key[d] : jobs[i].key[d] < key[d]) {
                key[d] = jobs[i].key[d];
                ext[d] = jobs[i].arg[d];
            }
        }
    }
    /* 2. octagon and filter */
    int64_t ox[8], oy[8], area2 = 0;
    for (int d = 0; d < 8; ++d) {
        ox[d] = (int64_t)pts[2 * ext[d]];
        oy[d] = (int64_t)pts[2 * ext[d] + 1];
    }
    for (int d = 0; d < 8; ++d) area2 += ox[d] * oy[(d + 1) & 7] - ox[(d + 1) & 7] * oy[d];
    for (int i = 0; i < t; ++i) {
        jobs[i].ox = area2 > 0 ? ox : NULL;
        jobs[i].oy = area2 > 0 ? oy : NULL;
        jobs[i].surv = surv + jobs[i].lo;
    }
    run_all(run_filter, jobs, t);
    int64_t m = 0;
    for (int i = 0; i < t; ++i) {   /* compact the chunks' survivors */
        if (surv + m != jobs[i].surv) memmove(surv + m, jobs[i].surv, (size_t)jobs[i].nsurv * sizeof(hpt));
        m += jobs[i].nsurv;
    }
    /* 3. order by (x, y, index): per-chunk sorts, then pairwise merges */
    tmp = (hpt*)malloc((size_t)(m > 0 ? m : 1) * sizeof(hpt));
    if (!tmp) goto done;
    int64_t bound[HH_MAX_THREADS + 1];
    int parts = (int64_t)t > m ? (int)(m > 0 ? m : 1) : t;
    for (int i = 0; i <= parts; ++i) bound[i] = m * i / parts;
    for (int i = 0; i < parts; ++i) {
        jobs[i].a = surv;
        jobs[i].m0 = bound[i];
        jobs[i].m1 = bound[i + 1];
    }
    run_all(run_sort, jobs, parts);
    hpt* src = surv;
    hpt* dst = tmp;
    for (int width = 1; width < parts; width *= 2) {
        int nj = 0;
        for (int i = 0; i < parts; i += 2 * width) {
            const int mid = i + width < parts ? i + width : parts;
            const int end = i + 2 * width < parts ? i + 2 * width : parts;
            jobs[nj].a = src;
            jobs[nj].b = dst;
            jobs[nj].m0 = bound[i];
            jobs[nj].m1 = bound[mid];
            jobs[nj].m2 = bound[end];
            ++nj;
        }
        run_all(run_merge, jobs, nj);
        hpt* s = src;
        src = dst;
        dst = s;
    }
    /* the first of each equal-(x, y) run has the lowest index */
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (u > 0 && src[u - 1].x == src[i].x && src[u - 1].y == src[i].y) continue;
        src[u++] = src[i];
    }
    if (u <= 2) {
        for (int64_t i = 0; i < u; ++i) out_idx[i] = (int32_t)src[i].idx;
        result = u;
        goto done;
    }
    /* Andrew's chains (the lower and the upper chain together hold at most 2u points) */
    hpt* h = (hpt*)malloc((size_t)(2 * u + 1) * sizeof(hpt));
    if (!h) goto done;
    int64_t k = 0;
    for (int64_t i = 0; i < u; ++i) {   /* lower chain */
        while (k >= 2 && cross3(h[k - 2].x, h[k - 2].y, h[k - 1].x, h[k - 1].y, src[i].x, src[i].y) <= 0) --k;
        h[k++] = src[i];
    }
    const int64_t lower_len = k + 1;
    for (int64_t i = u - 2; i >= 0; --i) {   /* upper chain */
        while (k >= lower_len && cross3(h[k - 2].x, h[k - 2].y, h[k - 1].x, h[k - 1].y, src[i].x, src[i].y) <= 0) --k;
        h[k++] = src[i];
    }
    --k;   /* the last point repeats the first */
    for (int64_t i = 0; i < k; ++i) out_idx[i] = (int32_t)h[i].idx;
    free(h);
    result = k;
done:
    free(tmp);
    free(surv);
    free(jobs);
    return result;
}
