/*
 * ch.h -- C ABI of the GB300 convex-hull library (libconvhull.so).
 *
 * The library computes the 2-D convex hull of a point set on one GPU with the
 * filtering method of GPU heaphull (Keith, Ferrada, Navarro; Alg. 1 and
 * Alg. 2): find the 8 directional extreme points, discard every point
 * strictly inside the octagon they span, sort the survivors of each of the
 * four corner queues, and build the hull of the survivors on the device.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Points are AoS float32 pairs (x0, y0, x1, y1, ...).  Every coordinate must
 *   be an integer value in [0, 2^24) (the paper only says "floating point",
 *   Alg. 2; integer values keep every predicate exact in int64).  A
 *   coordinate outside that domain (fraction, negative, >= 2^24, NaN, Inf)
 *   is a DATA error: it is detected on the device and reported through the
 *   output count as CH_ERANGE (never by a trap or a fault).
 * - "device" pointers are CUDA device (or managed) memory of the current
 *   device; "host" pointers are ordinary or pinned host memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   ch_hull, ch_filter, ch_filter16 and ch_hull_noalloc are stream-ordered:
 *   they return as soon as the work is enqueued and never synchronise the
 *   host with the device, so a sequence of them can be captured in a CUDA
 *   graph (after ch_reserve, see below).  The calls that do wait for the
 *   device say so in their own comments: ch_hull_batched (it reads a k-byte
 *   flag array back, and the offsets when no host copy is given), ch_hull_host,
 *   ch_reserve, ch_release, ch_selftest_timeout and ch_profile_read.
 * - Return value: CH_OK when the work was enqueued, or a negative ch_status
 *   for an error the host can see at call time (null pointer, bad size or
 *   alignment, allocation or launch failure).  No C++ exception crosses the ABI.
 * - The caller owns every buffer it passes.  The library owns an internal
 *   workspace per (device, stream), grown on demand and freed by ch_release().
 *   Calls on the SAME stream share that workspace in stream order; calls on
 *   different streams use different workspaces and may overlap.
 */
#ifndef CONVHULL_CH_H
#define CONVHULL_CH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CH_OK = 0,
    CH_PENDING = 1,     /* ch_poll: request admitted, result not ready yet */
    CH_EINVAL = -1,     /* bad argument (null pointer, negative size, alignment) */
    CH_ERANGE = -2,     /* a coordinate is not an integer in [0, 2^24) */
    CH_ENOMEM = -3,     /* device or host allocation failed / budget exceeded */
    CH_ECUDA = -4,      /* a CUDA runtime call failed */
    CH_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    CH_EBUSY = -6       /* serving queue full; retry later */
} ch_status;

/* Largest point count of one hull (indices are int32). */
#define CH_MAX_POINTS ((int64_t)0x7FFFFFF0)

/*
 * ch_hull -- convex hull of n points (Alg. 1's problem: P[1..n] in, the h hull
 * points in counter-clockwise order out).
 *   pts      device, 8-byte aligned, n*2 float32 (x, y interleaved).
 *   n        0 <= n <= CH_MAX_POINTS.
 *   out_idx  device int32, capacity n (h <= n).  On success holds the indices
 *            of the strictly convex hull vertices, counter-clockwise, starting
 *            at the lexicographically smallest (x, then y) vertex; points in
 *            the interior of a hull edge are excluded; a vertex whose
 *            coordinates occur several times is named by its lowest index.
 *            All points collinear: [lex-min, lex-max]; all identical: [lowest index].
 *   out_n    device int64*: the device writes h, or a negative ch_status when
 *            the input holds a value outside the domain (CH_ERANGE) or a
 *            device wait timed out (CH_ETIMEOUT).
 * Returns CH_OK on enqueue.  On sparse data (few points outside the octagon)
 * the points are streamed once (8 bytes per point): the extremes and the
 * filter share one pass.  When most points survive that pass's filter (points
 * near a circle, Table V) a second streaming pass classifies every point.  The
 * hull stage touches only the survivors.
 */
int ch_hull(const float* pts, int64_t n, int32_t* out_idx, int64_t* out_n, void* stream);

/*
 * ch_hull_batched -- k independent hulls in one set of launches.
 *   pts      device, 8-byte aligned, the k point sets packed back to back.
 *   offsets  device int64[k+1]: set i is points [offsets[i], offsets[i+1]);
 *            offsets[0] == 0, non-decreasing, each set <= CH_MAX_POINTS.
 *   k        0 <= k <= 2^20.
 *   out_idx  device int32, capacity offsets[k]; hull i is written to
 *            out_idx[offsets[i] .. offsets[i] + out_n[i]) as LOCAL indices
 *            (relative to offsets[i]), same order rules as ch_hull.
 *   out_n    device int64[k]: hull sizes, or a negative ch_status per set.
 *   host_offsets  optional HOST copy of offsets (NULL allowed): lets the
 *            library size its launches without reading the device array.
 * Each result equals ch_hull on that set alone.  The batch's points are
 * streamed as one array (extremes, then filter); dense sets of at least 32768
 * points are filtered by a star polygon of their own points (Table V's
 * worst case); see ch_batched_counters.
 * Shape of the streamed per-point kernels (threads per block x points per
 * lane, a warp tile being 32 x points per lane): picked by an autotuner per
 * (device name, SM count, floor log2 of offsets[k], floor log2 of k).  The first call of such a size
 * class times every compiled shape on that call's batch (the call blocks
 * meanwhile); the result is kept in memory and, when the environment variable
 * CH_TUNE_CACHE names a file, in that JSON file, read at the first lookup.
 * CH_BLOCK and CH_PPT (or CH_TILE = CH_BLOCK x CH_PPT) name a shape directly;
 * one that is not compiled makes the call return CH_EINVAL.  The device work
 * is launched as a CUDA graph that is updated in place from call to call
 * (per device and stream); the call reads a k-byte flag array back before it
 * returns (it synchronises the stream).
 */
int ch_hull_batched(const float* pts, const int64_t* offsets, int32_t k,
                    int32_t* out_idx, int64_t* out_n, const int64_t* host_offsets,
                    void* stream);

/*
 * ch_batched_counters -- what the most recent ch_hull_batched on `stream`
 * (current device) did per set, for measurement and tests: for set i,
 *   out[4 i]      records handed to the hull stage (the filter's survivors,
 *                 the chain end points included),
 *   out[4 i + 1]  vertices of the star polygon that filtered the set (0 when
 *                 none: a sparse set, a set under 32768 points, or a polygon
 *                 that failed its checks),
 *   out[4 i + 2]  the set's status (CH_OK or a negative ch_status),
 *   out[4 i + 3]  hull stage: 0 one block, 1 the bucketed path, 2 the
 *                 single-hull path.
 * k must equal that call's k; out holds 4 k values.  Returns 4 (values per
 * set).  Synchronises the stream.  CH_EINVAL when no batched call of k sets
 * ran on that stream (or out is NULL).
 */
int ch_batched_counters(void* stream, int32_t k, int64_t* out);

/*
 * ch_batched_config -- the tile shape ch_hull_batched uses on the current
 * device for a batch of total_points points in k >= 1 sets: *threads and
 * *per (points per lane) from CH_BLOCK / CH_PPT / CH_TILE, else from the
 * autotuner's choice for that size class; both 0 when it has not been tuned
 * yet.  CH_EINVAL for bad arguments or an environment shape that is not one
 * of the compiled shapes (128x16, 256x8, 256x16, 256x32, 512x8, 512x16).
 */
int ch_batched_config(int64_t total_points, int32_t k, int32_t* threads, int32_t* per);

/*
 * ch_filter -- the paper's GPUfilter (Alg. 2) on its own.
 *   out_ext8     device int32[8]: indices of the extreme points in the order
 *                W, SW, S, SE, E, NE, N, NW (argmin x, argmin x+y, argmin y,
 *                argmax x-y, argmax x, argmax x+y, argmax y, argmin x-y;
 *                lowest index on ties; Sec. 3 finds the last four by minimum
 *                Manhattan distance to the bounding-box corners, which selects
 *                the same points).  Entries are -1 when n == 0.
 *   out_labels   device uint8[n] or NULL: the array Q of Alg. 2; 0 when the
 *                point is strictly inside the octagon W..NW (or in no queue),
 *                else its queue 1..4: 1 = strictly right of W->S, 2 = right of
 *                S->E, 3 = right of E->N, 4 = right of N->W (first match).
 *   out_counts4  device int64[4] or NULL: number of points in each queue, or
 *                all four set to a negative ch_status on a data error.
 */
int ch_filter(const float* pts, int64_t n, int32_t* out_ext8, uint8_t* out_labels,
              int64_t* out_counts4, void* stream);

/*
 * ch_filter_manhattan -- ch_filter with the extremes found the way Sec. 3
 * finds them: a first streaming kernel reduces the axis extremes (W, E, S,
 * N, i.e. the bounding box), a second one the point of minimum Manhattan
 * distance to each corner of that box (SW, SE, NE, NW); lowest index on
 * ties.  Every point lies in the box, so those are the argmin / argmax of
 * x + y and x - y that ch_filter takes in its single pass: the outputs are
 * identical (same arguments, layouts and errors as ch_filter), but the input
 * is read twice before the labels.  Kept to measure the fused pass against
 * the paper's two-kernel form.
 */
int ch_filter_manhattan(const float* pts, int64_t n, int32_t* out_ext8, uint8_t* out_labels,
                        int64_t* out_counts4, void* stream);

/*
 * ch_filter16 -- ch_filter with a 16-direction polygon in place of the
 * octagon: the filter over a convex polygon of 16 extreme points that the
 * paper cites among related work (Sec. 2), with Alg. 2's rules.  The paper
 * gives no directions; they are the octagon's 8 and the 8 integer directions
 * between them, in counter-clockwise order from W:
 *   (-1,0) W, (-2,-1), (-1,-1) SW, (-1,-2), (0,-1) S, (1,-2), (1,-1) SE,
 *   (2,-1), (1,0) E, (2,1), (1,1) NE, (1,2), (0,1) N, (-1,2), (-1,1) NW,
 *   (-2,1).
 *   pts          as ch_filter (device, 8-byte aligned, integers in [0, 2^24)).
 *   out_ext16    device int32[16]: for direction k = (a, b) the index of the
 *                point maximising a x + b y, lowest index on ties (the even
 *                entries equal ch_filter's W, SW, ..., NW).  All -1 when
 *                n == 0 or on a data error.
 *   out_labels   device uint8[n] or NULL: 0 when the point is strictly inside
 *                the polygon of those 16 points (strictly left of every edge
 *                of non-zero length; a polygon of zero area discards nothing)
 *                or in no queue, else its queue 1..4 by ch_filter's
 *                quadrilateral rule over W, S, E, N.
 *   out_counts4  device int64[4] or NULL: points per queue, or all four set
 *                to CH_ERANGE when a coordinate is outside the domain.
 * Stream-ordered, no host synchronisation; uses the stream's workspace (as
 * ch_hull).  Returns CH_OK on enqueue or a negative status for bad arguments
 * (CH_EINVAL) or a launch error (CH_ECUDA).
 */
int ch_filter16(const float* pts, int64_t n, int32_t* out_ext16, uint8_t* out_labels,
                int64_t* out_counts4, void* stream);

/*
 * ch_hull_host -- ch_hull on HOST buffers: copies pts (host, n*2 float32) to
 * the device, computes the hull, copies the result back and waits for it.
 * Writes h (or a negative status) to *out_n and the indices to out_idx (host,
 * capacity n).  Returns CH_OK or a negative status.  Blocking.
 */
int ch_hull_host(const float* pts, int64_t n, int32_t* out_idx, int64_t* out_n, void* stream);

/* Largest point count of ch_hull_noalloc. */
#define CH_NOALLOC_MAX_POINTS ((int64_t)8000)

/*
 * ch_hull_noalloc -- ch_hull for at most CH_NOALLOC_MAX_POINTS points that
 * allocates nothing.  The paper has no counterpart; it exists for callers
 * that cannot let the library allocate device memory: code that must keep
 * within a device-memory budget fixed up front, or a latency-critical loop
 * that cannot pay the device-wide synchronisation cudaMalloc may imply
 * (ch_hull grows its workspace the first time it sees a size).
 *   pts      device, 8-byte aligned, n*2 float32 (same domain as ch_hull).
 *   n        0 <= n <= CH_NOALLOC_MAX_POINTS; larger n returns CH_EINVAL and
 *            enqueues nothing.
 *   out_idx  device int32[n], 4-byte aligned; out_n device int64 (8-byte
 *            aligned): the same result as ch_hull (h indices, CCW from the
 *            lexicographically smallest vertex; or CH_ERANGE on bad data).
 * The whole hull runs in one thread block.  Its global scratch (about 100 KB)
 * is one fixed array in the library's static device memory; the first call on
 * a device looks up that array's address and sets the kernel's shared-memory
 * limit, so make that first call before any stream capture.  The look-up is
 * kept per device and CUDA context: after the context is re-created (e.g. by
 * cudaDeviceReset) the next call repeats it.  Nothing in the
 * scratch needs to start at zero.  Calls that overlap in time (other streams
 * or host threads) share the scratch and race: the caller orders them.
 * Returns CH_OK when enqueued, CH_EINVAL or CH_ECUDA otherwise.
 */
int ch_hull_noalloc(const float* pts, int64_t n, int32_t* out_idx, int64_t* out_n, void* stream);

/*
 * ch_reserve -- grow the workspace of `stream` on the current device for
 * hulls of up to n points (batched: n = total points, k sets).  Call it before
 * capturing ch_hull / ch_hull_batched into a CUDA graph: allocation is not
 * allowed during capture.  Blocking (may synchronise `stream`).
 */
int ch_reserve(int64_t n, int32_t k, void* stream);

/*
 * ch_hull_counters -- what the most recent ch_hull on `stream` (current
 * device) did, for measurement and tests (ch_filter shares the control block
 * these come from, so after it they describe the filter): writes up to `cap` of
 *   out[0]  raw survivors of the fused streaming pass (points it could not
 *           discard against the sample's polygon),
 *   out[1]  sort records handed to the hull stage (the chain end points
 *           included): the survivors of the filter,
 *   out[2]  0 when one streaming pass did the extremes and the filter, 1 when
 *           a second pass classified every point,
 *   out[3]  hull stage: 0 finished by one block (few records), 1 bucketed
 *           chains, 2 the radix-sort fallback,
 *   out[4]  the call's status (CH_OK or the negative code it reported),
 *   out[5]  vertices of the star polygon that filtered dense data (0 when
 *           the call built none)
 * and returns how many counters exist (6).  Synchronises the stream.
 * CH_EINVAL when no hull ran on that stream (or out is NULL).
 */
int ch_hull_counters(void* stream, int64_t* out, int cap);

/* Bytes of workspace ch_hull needs for n points. */
size_t ch_workspace_bytes(int64_t n);

/* Free every workspace of every device (synchronises the streams involved). */
int ch_release(void);

/*
 * ch_selftest_timeout -- test support for failure detection: runs one of the
 * library's bounded device waits on a condition that never comes true
 * (which = 0: the radix-sort look-back poll on a flag nothing sets; 1: the
 * bulk-copy barrier wait with no copy issued).  The wait gives up after its
 * limit (well under a second) and the kernel returns; nothing traps or
 * faults and the context stays usable.  Returns the status the device
 * recorded, CH_ETIMEOUT when the wait gave up as designed; CH_EINVAL for a
 * bad `which`; CH_ENOMEM / CH_ECUDA for allocation or launch failures.
 * Synchronises `stream`.
 */
int ch_selftest_timeout(int which, void* stream);

/* Static text for a status code. */
const char* ch_strerror(int status);

/*
 * Device-timed kernel statistics.  When enabled, the library records CUDA
 * events around each kernel it launches, on the launching stream.
 * ch_profile_read synchronises those events and returns, for up to `cap`
 * kernels, the name, the number of launches and the summed milliseconds;
 * the return value is the number of distinct kernels (may exceed cap).
 */
int ch_profile_enable(int on);
int ch_profile_reset(void);
int ch_profile_read(const char** names, int64_t* launches, double* total_ms, int cap);

/*
 * Serving (continuous batching).  A server owns a device memory pool of
 * budget_bytes on `device` (its arena and the single-hull workspaces of its
 * batch streams; each stream's batched workspace comes on top) and an engine
 * thread with its own streams.  ch_submit queues the request without blocking
 * and without copying it: it returns CH_OK with a ticket, or CH_EBUSY when
 * the admission queue is full, or CH_ENOMEM when the request can never fit
 * the budget.  The server copies the points to the device when the request
 * is admitted into a batch (as memory frees up, together with the requests
 * that arrived meanwhile), so the host buffer pts_host must stay valid and
 * unchanged until ch_poll has answered for the ticket with anything but
 * CH_PENDING; pinned host memory avoids a staging copy in the driver.
 * ch_poll returns CH_PENDING, or CH_OK after copying the h result indices to
 * out_idx_host (capacity cap) and setting *out_n (the request's ticket is
 * then retired), or a negative status (CH_EINVAL for an unknown ticket).
 * ch_server_stats fills p50/p99 request latency in ms and served points/s.
 */
int ch_server_create(size_t budget_bytes, int device, void** srv);
int ch_submit(void* srv, const float* pts_host, int64_t n, uint64_t* ticket);
int ch_poll(void* srv, uint64_t ticket, int32_t* out_idx_host, int64_t cap, int64_t* out_n);
int ch_server_stats(void* srv, double* p50_ms, double* p99_ms, double* points_per_s,
                    int64_t* completed);
/*
 * ch_server_trace -- the server's retired batches, in order, 8 values each:
 * formation time (ms since the first submission), requests, points, time
 * of the host-to-device copies, of the batched hull with its result counts
 * back, of the index copies back (device time, CUDA events on the batch's
 * stream, ms), host time from formation to retirement (ms), and the sets
 * the batched kernels left to the single-hull path.  Writes up to cap
 * batches to out (8 cap doubles; out may be NULL when cap == 0) and returns
 * how many batches were traced (at most 2^20 are kept).
 */
int ch_server_trace(void* srv, double* out, int64_t cap);
int ch_server_destroy(void* srv);

#ifdef __cplusplus
}
#endif
#endif /* CONVHULL_CH_H */
