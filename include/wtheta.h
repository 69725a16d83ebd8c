/*
 * wtheta.h -- C ABI of libwtheta: exact angular pair counts (DD, DR, RR) and
 * the Landy-Szalay estimate of the two-point angular correlation function
 * w(theta), on one NVIDIA GB300 (sm_103a).
 *
 * The computation is the one stated in Sec. 2 of "Cosmological calculations
 * on the GPU" (Bard, Bellis, Allen, Yepremyan, Kratochvil; arXiv:1208.3658):
 * for every pair of galaxies, the angular separation (App. A) is binned into
 * a histogram between user-set limits (Sec. 2.1); DD and RR count each
 * unordered pair of one catalogue once, with no self pairs (n(n-1)/2 pairs),
 * DR counts every data-random pair (n n_r pairs), and Eq. 2 combines them.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: WTHETA_OK (0) or a negative WTHETA_E* code.  Nothing is
 *    written to outputs when a call fails argument validation.
 *  - Angles are FP64 degrees.  Catalogues are interleaved FP64
 *    [ra_0, dec_0, ra_1, dec_1, ...], RA any finite value, |Dec| <= 90.
 *  - Bin edges e_0 < e_1 < ... < e_K (K = n_bins, 1 <= K <= 256) are FP64
 *    degrees in [0, 180], host memory.  A pair with separation theta lands in
 *    slot 0 (underflow) if theta < e_0, slot k (1..K) if
 *    e_{k-1} <= theta < e_k, slot K+1 (overflow) if theta >= e_K.  The
 *    comparison is made exactly on the squared chord
 *    s = |a - b|^2 of the FP64 unit vectors, evaluated
 *    ((dx*dx + dy*dy) + dz*dz) with IEEE round-to-nearest and no fused
 *    operations, against c_k = 4 sin^2(e_k pi / 360) computed on the host.
 *    Counts are exact for that predicate.
 *  - Count arrays have K+2 uint64 slots (underflow, bins 1..K, overflow).
 *  - Device pointers are borrowed: the library never frees them, and they
 *    must be on the device that is current when the call is made.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device outputs are written asynchronously on it; the caller
 *    synchronises before reading them.  Scratch memory is taken from the
 *    device's stream-ordered pool on the same stream and returned on it.
 *  - Problems only the device can see (non-finite coordinates, |Dec| > 90,
 *    non-unit vectors) set bits in a sticky per-device error word, read and
 *    cleared by wtheta_get_error().  The counts of such a call are undefined.
 */
#ifndef WTHETA_H
#define WTHETA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define WTHETA_OK 0
#define WTHETA_EINVAL (-1)   /* bad size, pointer, edge array or option      */
#define WTHETA_ENOMEM (-2)   /* device or host allocation failed             */
#define WTHETA_ECUDA (-3)    /* a CUDA runtime call failed                   */
#define WTHETA_ETIMEOUT (-4) /* a bounded device or host wait gave up        */
#define WTHETA_EBUDGET (-5)  /* a request does not fit the memory budget     */
#define WTHETA_EDEVICE (-6)  /* the device error word is non-zero            */
#define WTHETA_ESIZE (-7)    /* input larger than a fixed-capacity entry point takes */
#define WTHETA_EBUSY (-8)    /* the object is in a state that forbids the call */
#define WTHETA_ECANCELED (-9) /* the request was cancelled before it ran      */

/* bits of the device error word (wtheta_get_error) */
#define WTHETA_DERR_NONFINITE 1u  /* an input coordinate is NaN or infinite  */
#define WTHETA_DERR_DEC_RANGE 2u  /* |Dec| > 90 degrees                      */
#define WTHETA_DERR_NOT_UNIT 4u   /* an xyz input is not a unit vector       */
#define WTHETA_DERR_LABEL 8u      /* a region label outside [0, n_regions)  */

/* ---- binning modes (Sec. 2.1: evenly spaced, natural-log, base-10 log) -- */
#define WTHETA_BINS_LINEAR 0
#define WTHETA_BINS_LN 1
#define WTHETA_BINS_LOG10 2

/* Message for a status code (static string, never NULL). */
const char* wtheta_strerror(int status);

/*
 * Bin edges for the three binning modes of Sec. 2.1 (user-set low and high
 * limits; evenly spaced, logarithmic or base-10 logarithmic widths).
 *   LINEAR: e_k = lo + k (hi - lo)/K
 *   LN:     e_k = lo exp(k ln(hi/lo)/K)
 *   LOG10:  e_k = lo 10^(k log10(hi/lo)/K)
 * with e_0 = lo and e_K = hi exactly.  The two logarithmic modes give the
 * same geometric edges up to rounding; the base names how the width is stated.
 * lo_deg >= 0 (> 0 for the log modes), hi_deg in (lo_deg, 180].
 * edges_out: host, K+1 doubles, written.  EINVAL on bad limits or K.
 */
int wtheta_edges(double lo_deg, double hi_deg, int32_t n_bins, int32_t mode,
                 double* edges_out);

/*
 * Squared-chord edges c_k = 4 sin^2(e_k pi/360) (App. A geometry: the chord
 * between unit vectors at angle theta is 2 sin(theta/2)).  These are the FP64
 * thresholds every count compares against.  Host in, host out (K+1 doubles).
 * EINVAL if the edges are not strictly increasing within [0, 180].
 */
int wtheta_chord2_edges(const double* edges_deg, int32_t n_bins, double* c_out);

/*
 * The FP32 screening thresholds the counting kernel uses (host only; exposed
 * so the guard band can be tested).  For each edge k, [lo_bits[k], hi_bits[k]]
 * is an interval of FP32 bit patterns (non-negative floats order like their
 * bits) around the FP32 edge: an FP32 squared chord below lo_bits[k] is
 * certainly below c_k in FP64 and one above hi_bits[k] certainly at or above
 * it; anything inside is recomputed in FP64.  The half-width bounds the
 * rounding of the unit vectors to FP32 and of the FP32 evaluation
 * d = a - b, s = fma(dz, dz, fma(dy, dy, dx*dx)).  All outputs host, K+1.
 */
int wtheta_guard_band(const double* edges_deg, int32_t n_bins, uint32_t* lo_bits,
                      uint32_t* hi_bits, double* half_width);

/*
 * Exact pair counts between two catalogues (Sec. 2): the DD/RR auto count or
 * the DR cross count, on the GPU.
 *   ra_dec_a, ra_dec_b: device, interleaved FP64 degrees, n_a / n_b points.
 *   is_auto = 1: ra_dec_b must be NULL or equal to ra_dec_a, n_b == n_a or 0;
 *     every unordered pair i < j of catalogue a is counted once, no self
 *     pairs: the slots sum to n_a (n_a - 1) / 2.
 *   is_auto = 0: all n_a n_b ordered pairs (i in a, j in b): the slots sum to
 *     n_a n_b.  Coincident points (theta = 0) are pairs like any other.
 *   bin_edges_deg: host, K+1 doubles (see the conventions above).
 *   counts: device, K+2 uint64, overwritten.
 * RA/Dec are converted to FP64 unit vectors on the device (CUDA's sin/cos,
 * which may differ from a host libm in the last place).  n = 0 gives all-zero
 * counts.  EINVAL on bad arguments, ENOMEM, ECUDA.
 */
int wtheta_count(const double* ra_dec_a, int64_t n_a, const double* ra_dec_b,
                 int64_t n_b, const double* bin_edges_deg, int32_t n_bins,
                 int32_t is_auto, uint64_t* counts, void* stream);

/*
 * As wtheta_count, from caller-supplied FP64 unit vectors instead of RA/Dec.
 *   xyz_a, xyz_b: device, SoA: x[0..n), y[0..n), z[0..n) (3n doubles).
 * Counts are a pure function of these bits and the edges.
 */
int wtheta_count_xyz(const double* xyz_a, int64_t n_a, const double* xyz_b,
                     int64_t n_b, const double* bin_edges_deg, int32_t n_bins,
                     int32_t is_auto, uint64_t* counts, void* stream);

/*
 * Sharding one count over several GPUs (or processes): the pair matrix is
 * split into n_shards contiguous ranges of rows (points of catalogue a, in
 * input order) holding equal numbers of pairs, up to one row.  A shard's
 * counts are exact for its pairs, overflow slot included, so the counts of
 * all shards add up (one sum-reduction of K+2 integers) to those of
 * wtheta_count.  The paper's summary notes that a straightforward division
 * of the data set lets the code run on clusters of independent GPUs.
 *
 * wtheta_shard_rows: host only; [*row_begin, *row_end) of shard (0-based).
 * wtheta_count_shard: as wtheta_count, for the shard's pairs only: rows
 *   [r0, r1) against all of b (cross), or, for auto counts, the pairs i < j
 *   with i in [r0, r1).
 */
int wtheta_shard_rows(int64_t n_a, int64_t n_b, int32_t is_auto, int32_t shard,
                      int32_t n_shards, int64_t* row_begin, int64_t* row_end);
int wtheta_count_shard(const double* ra_dec_a, int64_t n_a, const double* ra_dec_b,
                       int64_t n_b, const double* bin_edges_deg, int32_t n_bins,
                       int32_t is_auto, int32_t shard, int32_t n_shards, uint64_t* counts,
                       void* stream);

/*
 * Contiguous split of n_rows weighted rows among n_shards: shard s gets rows
 * [*row_begin, *row_end), the boundary before shard s being the first row
 * whose prefix weight (the sum of the weights of the rows before it) reaches
 * s/n_shards of the total; with all weights zero the rows are split evenly by
 * number.  The ranges of shards 0..n_shards-1 partition [0, n_rows).  Host
 * only.  weights: host, n_rows uint64.  EINVAL on bad arguments.
 */
int wtheta_shard_weights(const uint64_t* weights, int64_t n_rows, int32_t shard,
                         int32_t n_shards, int64_t* row_begin, int64_t* row_end);

/* Tuning knobs of the counting kernel; zero fields mean "choose". */
typedef struct wtheta_tune {
    int32_t threads;           /* threads per block: 64, 128 or 256           */
    int32_t points_per_thread; /* A points held in registers per thread: 8 or 16 */
    int32_t hist_mode;         /* 1: private per-thread histograms, plain add;
                                  2: per-warp histograms, warp-aggregated atomics;
                                  3: private per-thread histograms, shared atomic add;
                                  4: per-warp histograms, shared atomic add (lanes on
                                     one word merged by the hardware)              */
    int32_t j_per_screen;      /* B points per screening test: 1 or 2          */
    int32_t deferred;          /* 1: bin in-range pairs as they are screened;
                                  2: note screened steps, recompute and bin after */
    int32_t blocks_per_sm;     /* resident blocks per SM the grid is sized for */
    int32_t skip_far;          /* 1: skip tile pairs that bounding caps show to lie
                                  wholly beyond the top edge (exact: their pairs are
                                  overflow); 2: evaluate every tile pair; 0: skip
                                  when the tile pairs fill more than two waves of
                                  the launch                                      */
    int32_t span_bins;         /* 1: settle a thread's A points against a chunk of
                                  32 B points in one slot, or by one compare per pair
                                  against a single edge, when the bounding spheres
                                  of the two groups allow it (exact); 2: bin every
                                  pair through the table                          */
} wtheta_tune;

/* statistics slots accumulated by wtheta_count_ex (uint64 each) */
#define WTHETA_STAT_PAIRS 0     /* pairs whose squared chord was computed,
                                   tile padding included                      */
#define WTHETA_STAT_RECHECK 1   /* pairs recomputed in FP64 (guard band)      */
#define WTHETA_STAT_TILES 2     /* tile pairs evaluated                       */
#define WTHETA_STAT_SKIPPED 3   /* tile pairs skipped as wholly out of range  */
#define WTHETA_STAT_SPAN 4      /* pairs settled per (A group, B chunk) span,
                                   without a table lookup per pair            */
#define WTHETA_NSTATS 5

/*
 * wtheta_count / wtheta_count_xyz with explicit tuning and statistics.
 *   coords_are_xyz: 0 = RA/Dec inputs (as wtheta_count), 1 = SoA unit vectors.
 *   tune: host, may be NULL.
 *   stats: device, WTHETA_NSTATS uint64, may be NULL; ADDED to (not zeroed).
 */
int wtheta_count_ex(const double* coords_a, int64_t n_a, const double* coords_b,
                    int64_t n_b, int32_t coords_are_xyz, const double* bin_edges_deg,
                    int32_t n_bins, int32_t is_auto, uint64_t* counts,
                    const wtheta_tune* tune, uint64_t* stats, void* stream);

/*
 * The three counts of one w(theta) -- DD, DR and RR of a data catalogue and
 * its randoms -- in one call: each catalogue is converted and ordered once,
 * and the three counts are one persistent launch (far tile pairs skipped per
 * count).  Same inputs as wtheta_count_ex for each catalogue;
 *   counts: device, 3 x (K+2) uint64 (DD, DR, RR), overwritten;
 *   tune, stats: as wtheta_count_ex (stats added over the three counts).
 * Equal, slot for slot, to three wtheta_count_ex calls.
 */
int wtheta_count_wtheta(const double* coords_d, int64_t n_d, const double* coords_r,
                        int64_t n_r, int32_t coords_are_xyz, const double* bin_edges_deg,
                        int32_t n_bins, uint64_t* counts, const wtheta_tune* tune,
                        uint64_t* stats, void* stream);

/*
 * One shard of wtheta_count_wtheta, for one of n_shards GPUs or processes
 * (the paper's summary notes that a straightforward division of the data set
 * lets the code run on clusters of independent GPUs).  Every shard prepares
 * both whole catalogues (replicas: no data moves between shards) and splits
 * the tile rows of each count -- points of the count's first catalogue, in the
 * library's spatial order, 1024 (or 512) to a row -- into n_shards contiguous
 * ranges holding equal numbers of kept tile pairs (wtheta_shard_weights over
 * the tile pairs whose bounding caps may meet below the top edge), so that
 * shards of a clustered survey get equal work rather than equal pair totals.
 * The shard counts the pairs whose first point lies in its rows; its 3 (K+2)
 * counts (DD, DR, RR) are exact for those pairs, overflow slot included, and
 * the counts of all shards add up, slot by slot (one sum-reduction of
 * 3 (K+2) integers, e.g. an all-reduce), to those of wtheta_count_wtheta.
 * The split is a deterministic function of the inputs, so every shard
 * computes the same one.  Synchronises stream once (the kept tile pairs per
 * row come to the host).  Other arguments as wtheta_count_wtheta; EINVAL
 * unless 0 <= shard < n_shards.
 */
int wtheta_count_wtheta_shard(const double* coords_d, int64_t n_d, const double* coords_r,
                              int64_t n_r, int32_t coords_are_xyz, const double* bin_edges_deg,
                              int32_t n_bins, int32_t shard, int32_t n_shards, uint64_t* counts,
                              const wtheta_tune* tune, uint64_t* stats, void* stream);

/*
 * Batched counts: the DD, DR and RR of many (data, randoms) catalogue pairs
 * sharing one edge set, in one persistent launch captured in a CUDA graph.
 * The paper's §4 motivates it: Monte-Carlo error estimates of w(theta) need
 * many mock catalogues counted exactly.  Every count of every pair becomes a
 * contiguous range of items (tile pairs) of one work queue, biggest count
 * first; the CTAs of one launch take items from a device cursor, so the
 * uneven catalogue sizes share the GPU without idle SMs.
 *
 *   cats: host array of n_cats entries; the pointers in them are device,
 *     interleaved FP64 RA/Dec degrees, borrowed for the plan's lifetime (each
 *     run reads their current contents).
 *   tune: NULL = autotune at plan time (kernel shape and histogram mode timed
 *     on a sample of this batch's work; results are cached per device for
 *     batches of similar size and bin count); else the given shape.
 *   stream: used for the plan-time preparation and autotuning.
 *   *plan: receives the plan; free it with wtheta_batch_free.
 * 1 <= n_cats <= 32768.  The plan owns its scratch (FP32/FP64 copies of every
 * catalogue), its work table and its graph.  The catalogues are prepared
 * together on every run, by a constant number of launches whatever n_cats:
 * one conversion into a single FP64 array, one spatial sort by (catalogue,
 * key), one gather into FP32 copies with each catalogue on tile boundaries,
 * one pass of chunk spheres and one of tile caps.
 */
typedef struct wtheta_catalog_pair {
    const double* data;
    int64_t n_data;
    const double* rand;
    int64_t n_rand;
} wtheta_catalog_pair;

typedef struct wtheta_plan wtheta_plan;

int wtheta_batch_plan(const wtheta_catalog_pair* cats, int32_t n_cats,
                      const double* bin_edges_deg, int32_t n_bins, const wtheta_tune* tune,
                      void* stream, wtheta_plan** plan);

/*
 * As wtheta_batch_plan, with the catalogues given either as RA/Dec
 * (coords_are_xyz = 0: interleaved FP64 degrees, converted on the device on
 * every run) or as FP64 unit vectors (coords_are_xyz = 1: SoA, x[0..n),
 * y[0..n), z[0..n) per catalogue), in which case the counts are a pure
 * function of those bits, like wtheta_count_xyz's.
 */
int wtheta_batch_plan_ex(const wtheta_catalog_pair* cats, int32_t n_cats, int32_t coords_are_xyz,
                         const double* bin_edges_deg, int32_t n_bins, const wtheta_tune* tune,
                         void* stream, wtheta_plan** plan);

/*
 * Runs a plan: one graph replay (the shared preparation of every catalogue,
 * the single pair-count launch, the overflow slots), then copies
 * the counts to counts: device, n_cats x 3 x (K+2) uint64, laid out
 * [cat][DD, DR, RR][slot].  Asynchronous on stream.
 */
int wtheta_batch_run(wtheta_plan* plan, uint64_t* counts, void* stream);

/* What a plan chose and holds (host struct filled by wtheta_batch_info). */
typedef struct wtheta_batch_info_t {
    wtheta_tune tune;          /* the kernel shape in use                    */
    int64_t n_items;           /* tile pairs in the work queue               */
    int64_t pairs;             /* algorithmic pairs of all counts            */
    int64_t evaluated_pairs;   /* pairs whose squared chord the last run
                                  computed (WTHETA_STAT_PAIRS; before the first
                                  run: all tile pairs); synchronises the device */
    int32_t n_counts;          /* 3 n_cats                                   */
    int32_t graph_kernels;     /* kernel launches per replay                 */
    float autotune_ms;         /* plan-time autotuning cost                  */
    int32_t autotuned;         /* 1 if the shape came from the autotuner     */
} wtheta_batch_info_t;

int wtheta_batch_info(const wtheta_plan* plan, wtheta_batch_info_t* info);

/* Releases a plan (synchronises its device work first). */
int wtheta_batch_free(wtheta_plan* plan);

/*
 * Serving: w(theta) requests of different sizes, counted with continuous
 * batching (the paper's §2.2 notes that overlapping transfers with kernels
 * matters for larger datasets).  A scheduler thread admits requests in
 * arrival order while their device copies fit under hbm_budget_bytes,
 * uploads and orders them on one stream while another counts, and runs
 * rounds: each round is one persistent pair-count launch over tile pairs of
 * every admitted request, so a request that arrives while others are counting
 * starts at the next round instead of waiting for them to finish.  Results
 * do not depend on how requests were mixed (integer counts).
 *
 *   WTHETA_REQ_AUTO:  data, rand -> DD, DR, RR and w = Eq. 2 (wtheta_ls);
 *   WTHETA_REQ_CROSS: data (D1), rand (R1), data2 (D2), rand2 (R2) ->
 *                     D1D2, D1R2, R1D2, R1R2 and w (wtheta_ls_cross).
 * Inputs are host arrays of interleaved FP64 RA/Dec degrees; submit copies
 * them, so the caller may reuse them at once.
 */
#define WTHETA_REQ_AUTO 0
#define WTHETA_REQ_CROSS 1

typedef struct wtheta_request {
    int32_t kind;
    const double* data;
    int64_t n_data;
    const double* rand;
    int64_t n_rand;
    const double* data2;    /* cross only */
    int64_t n_data2;
    const double* rand2;    /* cross only */
    int64_t n_rand2;
} wtheta_request;

/* request states reported by wtheta_server_request_info */
#define WTHETA_RS_QUEUED 0
#define WTHETA_RS_UPLOADING 1
#define WTHETA_RS_COUNTING 2
#define WTHETA_RS_FINISHING 3
#define WTHETA_RS_DONE 4
#define WTHETA_RS_FAILED 5

typedef struct wtheta_request_info {
    int32_t state;
    int32_t status;           /* WTHETA_OK or the error that failed it       */
    double t_submit;          /* seconds since the server was created        */
    double t_admit;
    double t_done;
    int64_t pairs;            /* algorithmic pairs of its counts             */
    int32_t n_counts;         /* 3 (auto) or 4 (cross)                        */
} wtheta_request_info;

typedef struct wtheta_server_stats_t {
    int64_t rounds;           /* pair-count launches so far                   */
    int64_t completed;        /* requests done                                */
    int64_t queued;           /* submitted, not yet admitted                  */
    int64_t active;           /* admitted, not yet done                       */
    int64_t items;            /* tile pairs counted                           */
    int64_t resident_bytes;   /* device memory held by admitted requests      */
    int64_t kernels;          /* kernel launches issued by the scheduler      */
} wtheta_server_stats_t;

typedef struct wtheta_server wtheta_server;

/* Starts a server for one edge set.  max_active: admitted requests at most
 * (0 = 1024).  tune: kernel shape (NULL = default). */
int wtheta_server_create(const double* bin_edges_deg, int32_t n_bins, size_t hbm_budget_bytes,
                         int32_t max_active, const wtheta_tune* tune, wtheta_server** server);

/* Queues a request; *req_id identifies it.  EBUDGET if it alone exceeds the
 * budget, EINVAL on bad arguments (fewer than 2 points in a catalogue). */
int wtheta_server_submit(wtheta_server* server, const wtheta_request* request, uint64_t* req_id);

/* Waits up to timeout_ms (0 = just look) for a request.  *done = 1 when it
 * has finished; then counts (host, n_counts x (K+2), may be NULL) and w (host,
 * K, may be NULL) are written.  ETIMEOUT if timeout_ms > 0 ran out. */
int wtheta_server_wait(wtheta_server* server, uint64_t req_id, int64_t timeout_ms, int32_t* done,
                       uint64_t* counts, double* w);

int wtheta_server_request_info(wtheta_server* server, uint64_t req_id, wtheta_request_info* info);

/* Cancels a request that is still queued (not yet admitted): it ends in
 * state WTHETA_RS_FAILED with status WTHETA_ECANCELED, and its wait returns
 * that status.  WTHETA_EBUSY once it has been admitted (its work is on the
 * device and runs to the end). */
int wtheta_server_cancel(wtheta_server* server, uint64_t req_id);

/* Forgets a finished request (frees its host copies). */
int wtheta_server_release(wtheta_server* server, uint64_t req_id);

int wtheta_server_stats(wtheta_server* server, wtheta_server_stats_t* stats);

/* Stops the scheduler, waits for the GPU, frees everything. */
int wtheta_server_destroy(wtheta_server* server);

/*
 * Allocation-free variant of wtheta_count_xyz (the paper has no counterpart).
 *
 * Some callers cannot let a library allocate device memory: a process whose
 * framework already owns the device's memory in its own pool (so a library
 * cudaMalloc fails or breaks its accounting), a server that reserves a fixed
 * memory budget up front, or a latency-bound loop that cannot afford an
 * allocation's implicit synchronisation.  This entry point allocates nothing:
 * it calls no cudaMalloc, cudaMallocAsync, cudaFree or allocating library
 * routine.  The caller passes the inputs and the output; the only scratch
 * (FP32 copies of both catalogues and a work cursor) lives in one fixed
 * device array inside libwtheta, 256 B + 16 B x WTHETA_NOALLOC_MAX_POINTS
 * (about 4 MiB), which every device that loads the library holds until the
 * process exits.
 *
 * Arguments, result and exactness are those of wtheta_count_xyz (same
 * kernels, same counts).  Limit: with n rounded up to a whole tile of
 * WTHETA_NOALLOC_TILE points, round_up(n_a) + round_up(n_b) (auto: round_up(n_a)
 * alone) must not exceed WTHETA_NOALLOC_MAX_POINTS; larger inputs return
 * WTHETA_ESIZE and nothing is launched.
 *
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call on each device before any stream capture.
 * A device reset (cudaDeviceReset) or anything else that unloads the
 * library's module from a device invalidates that address: do not call this
 * entry point on a device after resetting it.  Every call reuses the same array, which keeps
 * the previous call's contents (each call rewrites what it reads and clears
 * its cursor): calls whose work can overlap on the GPU, from several streams
 * or host threads, race on the array and give wrong counts, so serialise them.
 */
#define WTHETA_NOALLOC_MAX_POINTS 262144
#define WTHETA_NOALLOC_TILE 1024
int wtheta_count_xyz_noalloc(const double* xyz_a, int64_t n_a, const double* xyz_b,
                             int64_t n_b, const double* bin_edges_deg, int32_t n_bins,
                             int32_t is_auto, uint64_t* counts, void* stream);

/*
 * RA/Dec (device, interleaved FP64 degrees) -> FP64 unit vectors (device,
 * SoA 3n doubles): x = cos(dec) cos(ra), y = cos(dec) sin(ra), z = sin(dec).
 * The conversion every wtheta_count call makes; exposed for testing.
 */
int wtheta_radec_to_xyz(const double* ra_dec, int64_t n, double* xyz, void* stream);

/*
 * Synchronises stream, then reads and clears the calling device's sticky
 * error word into *code (0 = no problem; else WTHETA_DERR_* bits).
 */
int wtheta_get_error(void* stream, uint32_t* code);

/*
 * Instrumentation (the paper has no counterpart): number of CUDA kernels this
 * library has launched in the process so far, all devices and streams.
 */
uint64_t wtheta_kernel_launches(void);

/*
 * Landy-Szalay estimator, Eq. 2, w = (DD - 2 DR + RR) / RR, evaluated on
 * counts normalised by their pair totals (Sec. 2): dd = DD_k / (n_d(n_d-1)/2),
 * dr = DR_k / (n_d n_r), rr = RR_k / (n_r(n_r-1)/2), then
 * w_k = ((dd - 2 dr) + rr) / rr in FP64, for k = 1..K.
 *   DD, DR, RR: host, K+2 slots each (as produced by wtheta_count).
 *   w: host, K doubles.  Bins with RR_k = 0 give NaN.
 * Requires n_d >= 2, n_r >= 2.
 */
int wtheta_ls(const uint64_t* DD, const uint64_t* DR, const uint64_t* RR, int64_t n_d,
              int64_t n_r, int32_t n_bins, double* w);

/*
 * Cross-correlation form of the same estimator between catalogues 1 and 2
 * with their randoms: w = (d1d2 - d1r2 - r1d2 + r1r2) / r1r2, each count
 * normalised by the product of its catalogue sizes, evaluated in that order.
 * Host arrays of K+2 slots; w: host, K doubles.  Bins with R1R2_k = 0 give
 * NaN.
 */
int wtheta_ls_cross(const uint64_t* D1D2, const uint64_t* D1R2, const uint64_t* R1D2,
                    const uint64_t* R1R2, int64_t n_d1, int64_t n_d2, int64_t n_r1,
                    int64_t n_r2, int32_t n_bins, double* w);

/*
 * Other estimators over the same counts (the paper leaves the choice of
 * estimator to the user, Sec. 2), each on counts normalised as in wtheta_ls
 * (dd, dr, rr), for k = 1..K, in FP64:
 *   WTHETA_EST_LANDY_SZALAY   ((dd - 2 dr) + rr) / rr      (= wtheta_ls)
 *   WTHETA_EST_NATURAL        dd / rr - 1                   (Peebles-Hauser)
 *   WTHETA_EST_DAVIS_PEEBLES  dd / dr - 1
 *   WTHETA_EST_HAMILTON       (dd rr) / (dr dr) - 1
 * A bin whose denominator count is 0 gives NaN.  Host arrays of K+2 slots;
 * w: host, K doubles.  Requires n_d >= 2, n_r >= 2; EINVAL for an unknown
 * estimator.
 */
#define WTHETA_EST_LANDY_SZALAY 0
#define WTHETA_EST_NATURAL 1
#define WTHETA_EST_DAVIS_PEEBLES 2
#define WTHETA_EST_HAMILTON 3
int wtheta_estimate(const uint64_t* DD, const uint64_t* DR, const uint64_t* RR, int64_t n_d,
                    int64_t n_r, int32_t n_bins, int32_t estimator, double* w);

/*
 * Jackknife regions.  Sec. 4 of the paper points at error estimates of
 * w(theta) from many realisations; the delete-one jackknife draws them from
 * the survey itself, cut into R regions.  wtheta_count_regions counts DD, DR
 * and RR split by region pair, in one persistent launch:
 *   coords_d, coords_r: device, as wtheta_count_ex (RA/Dec degrees, or SoA
 *     unit vectors when coords_are_xyz = 1);
 *   labels_d, labels_r: device int32, the region of every point, in
 *     [0, n_regions); 1 <= n_regions <= 256 (a label outside sets
 *     WTHETA_DERR_LABEL in the device error word and counts as region 0);
 *   counts: device, 3 x R x R x (K+2) uint64, laid out [DD, DR, RR][a][b][slot]:
 *     DD and RR hold the pairs with one point in region a and the other in
 *     region b for a <= b (a = b: both in a) and zeros for a > b; DR holds
 *     the pairs of a data point in region a and a random point in region b;
 *   region_sizes: host, 2 x R int64 (points per region: data, then randoms).
 * Synchronises stream once (the region sizes decide the launch's layout).
 * Summing the region pairs gives wtheta_count's DD, DR and RR.
 */
int wtheta_count_regions(const double* coords_d, int64_t n_d, const int32_t* labels_d,
                         const double* coords_r, int64_t n_r, const int32_t* labels_r,
                         int32_t coords_are_xyz, const double* bin_edges_deg, int32_t n_bins,
                         int32_t n_regions, uint64_t* counts, int64_t* region_sizes,
                         void* stream);

/*
 * Delete-one jackknife of the Landy-Szalay w(theta) from region-pair counts
 * (host copies of wtheta_count_regions' outputs).  Sample k drops every pair
 * with a point in region k and the region's points from the pair totals:
 *   w: K doubles, the estimate from all regions (= wtheta_ls of the sums);
 *   w_jk: R x K doubles, sample k in row k;
 *   cov: K x K doubles, (R-1)/R sum_k (w_k - mean)(w_k - mean)^T.
 * Requires 2 <= R <= 256.
 */
int wtheta_jackknife(const uint64_t* counts, const int64_t* region_sizes, int32_t n_regions,
                     int32_t n_bins, double* w, double* w_jk, double* cov);

/*
 * Fault injection on the host, for tests of the failure paths: the device
 * allocation made after `after` more successful ones fails with
 * WTHETA_ENOMEM (after = 0: the next one); -1 turns it off.  No GPU work is
 * involved in the failure.  Process-wide.
 */
int wtheta_inject_alloc_failure(int32_t after);

/*
 * Measurement: the shared-memory atomic throughput of the current device,
 * for the pair kernel's second roofline (its histogram updates are shared
 * reductions).  One block of 1024 threads per SM issues red.shared.add.u32,
 * each thread to its own word (same_address = 0) or all to one word (1);
 * *per_sm_per_clock receives warp-wide reductions per SM per SM clock.
 * Synchronises the device.  Not part of the paper's method.
 */
int wtheta_probe_shared_atomics(int32_t same_address, double* per_sm_per_clock);

/*
 * Whole w(theta) from host catalogues: copies data and randoms to the device
 * on stream, counts DD, DR, RR, copies the counts back and applies
 * wtheta_ls.  Synchronises stream before returning.
 *   data, rand: host, interleaved FP64 degrees.
 *   counts_out: host, 3 (K+2) uint64 (DD, DR, RR), may be NULL.
 *   w_out: host, K doubles, may be NULL.
 */
int wtheta_correlate(const double* data, int64_t n_d, const double* rand, int64_t n_r,
                     const double* bin_edges_deg, int32_t n_bins, uint64_t* counts_out,
                     double* w_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WTHETA_H */
