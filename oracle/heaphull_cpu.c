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
 *      by (x, y, index): stable LSD radix passes on the 48-bit key
 *      x * 2^24 + y, every chunk counting and scattering its share of each
 *      pass (the survivors arrive in index order, so equal coordinates stay
 *      in index order); the first of each run of equal coordinates stays.
 *   4. Andrew's chains: each chunk of the sorted points builds its lower and
 *      upper chain, and one pass over the concatenated chunk chains gives
 *      the hull (the hull of a sorted list is the hull of its pieces' hulls,
 *      in order).
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

/* a survivor: key = x * 2^24 + y (orders by x, then y), and its index */
typedef struct {
    uint64_t key;
    int64_t idx;
} hpt;

static int64_t px(const hpt* p) { return (int64_t)(p->key >> 24); }
static int64_t py(const hpt* p) { return (int64_t)(p->key & 0xFFFFFFu); }

/* direction order W, SW, S, SE, E, NE, N, NW (counter-clockwise around the
 * hull); key d is minimised for W, SW, S, NW and maximised for SE, E, NE, N */
static int dir_max(int d) { return d >= 3 && d <= 6; }

/* an integer in [0, 2^24): the truncation is exact only for integers; NaN
 * fails the range test */
static int coord_ok(float v) { return v >= 0.0f && v < 16777216.0f && (float)(int32_t)v == v; }

static int64_t cross3(int64_t ox, int64_t oy, int64_t ax, int64_t ay, int64_t bx, int64_t by) {
    return (ax - ox) * (by - oy) - (ay - oy) * (bx - ox);
}

/* cross3 of three survivors */
static int64_t turn(const hpt* o, const hpt* a, const hpt* b) {
    return cross3(px(o), py(o), px(a), py(a), px(b), py(b));
}

/* ---------------------------------------------------------------------- */
typedef struct {
    const float* pts;
    int64_t lo, hi;
    int bad;
    int64_t key[8], arg[8];   /* step 1 */
    const int64_t* ea;        /* step 2: live octagon edges a x + b y + c (> 0: strictly left) */
    const int64_t* eb;
    const int64_t* ec;
    int ne;                   /*   their number; -1 = keep every point */
    hpt* surv;                /* step 2: this chunk's survivors */
    int64_t nsurv;
    const hpt* src;           /* step 3: one radix pass over src[m0, m1) into dst */
    hpt* dst;
    int sh;                   /*   digit shift */
    int64_t* cnt;             /*   this chunk's digit counts, then its scatter cursors */
    hpt* low;                 /* step 4: lower / upper chain of src[m0, m1) */
    hpt* up;
    int64_t nl, nu;
    int64_t m0, m1;
} job;

static void* run_extremes(void* arg) {
    job* j = (job*)arg;
    j->bad = 0;
    /* minima of x, x + y, y, x - y and maxima of x - y, x, x + y, y */
    int32_t wx = INT32_MAX, sws = INT32_MAX, sy = INT32_MAX, nwd = INT32_MAX;
    int32_t sed = INT32_MIN, ex = INT32_MIN, nes = INT32_MIN, ny = INT32_MIN;
    int64_t aw = -1, asw = -1, as = -1, anw = -1, ase = -1, ae = -1, ane = -1, an = -1;
    for (int64_t i = j->lo; i < j->hi; ++i) {
        const float fx = j->pts[2 * i], fy = j->pts[2 * i + 1];
        if (!coord_ok(fx) || !coord_ok(fy)) {
            j->bad = 1;
            return NULL;
        }
        const int32_t x = (int32_t)fx, y = (int32_t)fy, s = x + y, d = x - y;
        /* strict improvement keeps the lowest index */
        if (x < wx) { wx = x; aw = i; }
        if (s < sws) { sws = s; asw = i; }
        if (y < sy) { sy = y; as = i; }
        if (d > sed) { sed = d; ase = i; }
        if (x > ex) { ex = x; ae = i; }
        if (s > nes) { nes = s; ane = i; }
        if (y > ny) { ny = y; an = i; }
        if (d < nwd) { nwd = d; anw = i; }
    }
    const int32_t k[8] = {wx, sws, sy, sed, ex, nes, ny, nwd};
    const int64_t a[8] = {aw, asw, as, ase, ae, ane, an, anw};
    for (int d = 0; d < 8; ++d) {
        j->key[d] = j->hi > j->lo ? (int64_t)k[d] : (dir_max(d) ? INT64_MIN : INT64_MAX);
        j->arg[d] = a[d];
    }
    return NULL;
}

static void* run_filter(void* arg) {
    job* j = (job*)arg;
    int64_t m = 0;
    for (int64_t i = j->lo; i < j->hi; ++i) {
        const int64_t x = (int64_t)j->pts[2 * i], y = (int64_t)j->pts[2 * i + 1];
        int inside = j->ne >= 0;
        for (int e = 0; e < j->ne; ++e) inside &= j->ea[e] * x + j->eb[e] * y + j->ec[e] > 0;
        if (inside) continue;
        j->surv[m].key = ((uint64_t)x << 24) | (uint64_t)y;
        j->surv[m].idx = i;
        ++m;
    }
    j->nsurv = m;
    return NULL;
}

/* Step 3: stable LSD radix sort by key, RADIX_BITS per pass over the 48-bit
 * key, all chunks at once: each counts its digits, the counts become
 * (digit, chunk)-major offsets, and each chunk scatters its records in
 * order, so a pass is stable */
#define RADIX_BITS 12
#define RADIX_BUCKETS (1 << RADIX_BITS)
#define RADIX_PASSES ((48 + RADIX_BITS - 1) / RADIX_BITS)

static void* run_count(void* arg) {
    job* j = (job*)arg;
    memset(j->cnt, 0, RADIX_BUCKETS * sizeof(int64_t));
    for (int64_t i = j->m0; i < j->m1; ++i) j->cnt[(j->src[i].key >> j->sh) & (RADIX_BUCKETS - 1)]++;
    return NULL;
}

static void* run_scatter(void* arg) {
    job* j = (job*)arg;
    for (int64_t i = j->m0; i < j->m1; ++i) j->dst[j->cnt[(j->src[i].key >> j->sh) & (RADIX_BUCKETS - 1)]++] = j->src[i];
    return NULL;
}

/* Step 4: Andrew's lower chain (pop while not a left turn) and upper chain
 * (pop while not a right turn) of the sorted, distinct points src[m0, m1),
 * both in ascending order.  The hull of a sorted list is the hull of the
 * concatenated chains of its pieces, so the final pass runs over these. */
static void* run_chains(void* arg) {
    job* j = (job*)arg;
    int64_t nl = 0, nu = 0;
    for (int64_t i = j->m0; i < j->m1; ++i) {
        const hpt* p = &j->src[i];
        while (nl >= 2 && turn(&j->low[nl - 2], &j->low[nl - 1], p) <= 0) --nl;
        j->low[nl++] = *p;
        while (nu >= 2 && turn(&j->up[nu - 2], &j->up[nu - 1], p) >= 0) --nu;
        j->up[nu++] = *p;
    }
    j->nl = nl;
    j->nu = nu;
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
    hpt* up = NULL;
    hpt* h = NULL;
    int64_t* cnt = NULL;
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
    /* edge V_d -> V_d+1 as a x + b y + c = orient(V_d, V_d+1, p); zero-length
     * edges are skipped, an octagon of zero area keeps everything */
    int64_t ea[8], eb[8], ec[8];
    int ne = 0;
    for (int d = 0; d < 8; ++d) {
        const int f = (d + 1) & 7;
        const int64_t dx = ox[f] - ox[d], dy = oy[f] - oy[d];
        if (dx == 0 && dy == 0) continue;
        ea[ne] = -dy;
        eb[ne] = dx;
        ec[ne] = dy * ox[d] - dx * oy[d];
        ++ne;
    }
    for (int i = 0; i < t; ++i) {
        jobs[i].ea = ea;
        jobs[i].eb = eb;
        jobs[i].ec = ec;
        jobs[i].ne = area2 > 0 ? ne : -1;
        jobs[i].surv = surv + jobs[i].lo;
    }
    run_all(run_filter, jobs, t);
    int64_t m = 0;
    for (int i = 0; i < t; ++i) {   /* compact the chunks' survivors */
        if (surv + m != jobs[i].surv) memmove(surv + m, jobs[i].surv, (size_t)jobs[i].nsurv * sizeof(hpt));
        m += jobs[i].nsurv;
    }
    /* 3. order by (x, y, index): parallel stable radix passes over the key
     * (the survivors are in index order, so ties stay in index order) */
    tmp = (hpt*)malloc((size_t)(m > 0 ? m : 1) * sizeof(hpt));
    cnt = (int64_t*)malloc((size_t)t * RADIX_BUCKETS * sizeof(int64_t));
    if (!tmp || !cnt) goto done;
    int64_t bound[HH_MAX_THREADS + 1];
    int parts = (int64_t)t > m ? (int)(m > 0 ? m : 1) : t;
    for (int i = 0; i <= parts; ++i) bound[i] = m * i / parts;
    hpt* src = surv;
    hpt* dst = tmp;
    for (int pass = 0; pass < RADIX_PASSES; ++pass) {
        for (int i = 0; i < parts; ++i) {
            jobs[i].src = src;
            jobs[i].dst = dst;
            jobs[i].sh = RADIX_BITS * pass;
            jobs[i].cnt = cnt + (size_t)i * RADIX_BUCKETS;
            jobs[i].m0 = bound[i];
            jobs[i].m1 = bound[i + 1];
        }
        run_all(run_count, jobs, parts);
        int64_t run = 0;
        for (int d = 0; d < RADIX_BUCKETS; ++d)
            for (int i = 0; i < parts; ++i) {
                const int64_t c = jobs[i].cnt[d];
                jobs[i].cnt[d] = run;
                run += c;
            }
        run_all(run_scatter, jobs, parts);
        hpt* sw = src;
        src = dst;
        dst = sw;
    }
    /* the first of each equal-(x, y) run has the lowest index */
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (u > 0 && src[u - 1].key == src[i].key) continue;
        src[u++] = src[i];
    }
    if (u <= 2) {
        for (int64_t i = 0; i < u; ++i) out_idx[i] = (int32_t)src[i].idx;
        result = u;
        goto done;
    }
    /* 4. Andrew's chains: per chunk in parallel, then one pass over the
     * concatenated chunk chains (dst is free scratch now) */
    up = (hpt*)malloc((size_t)u * sizeof(hpt));
    h = (hpt*)malloc((size_t)(2 * u + 1) * sizeof(hpt));
    if (!up || !h) goto done;
    parts = (int64_t)t > u ? (int)u : t;
    for (int i = 0; i <= parts; ++i) bound[i] = u * i / parts;
    for (int i = 0; i < parts; ++i) {
        jobs[i].src = src;
        jobs[i].low = dst + bound[i];
        jobs[i].up = up + bound[i];
        jobs[i].m0 = bound[i];
        jobs[i].m1 = bound[i + 1];
    }
    run_all(run_chains, jobs, parts);
    int64_t nl = 0, nu = 0;   /* compact the chunk chains, in chunk order */
    for (int i = 0; i < parts; ++i) {
        memmove(dst + nl, jobs[i].low, (size_t)jobs[i].nl * sizeof(hpt));
        memmove(up + nu, jobs[i].up, (size_t)jobs[i].nu * sizeof(hpt));
        nl += jobs[i].nl;
        nu += jobs[i].nu;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < nl; ++i) {   /* lower chain, lexicographic minimum to maximum */
        while (k >= 2 && turn(&h[k - 2], &h[k - 1], &dst[i]) <= 0) --k;
        h[k++] = dst[i];
    }
    const int64_t lower_len = k + 1;
    for (int64_t i = nu - 2; i >= 0; --i) {   /* upper chain, back to the minimum */
        while (k >= lower_len && turn(&h[k - 2], &h[k - 1], &up[i]) <= 0) --k;
        h[k++] = up[i];
    }
    --k;   /* the last point repeats the first */
    for (int64_t i = 0; i < k; ++i) out_idx[i] = (int32_t)h[i].idx;
    result = k;
done:
    free(h);
    free(up);
    free(cnt);
    free(tmp);
    free(surv);
    free(jobs);
    return result;
}
