// Serving w(theta) requests with continuous batching.
//
// A request is one w(theta): DD, DR, RR of a data catalogue and its randoms
// (Eq. 2), or the four counts of a cross-correlation between two catalogues
// and their randoms.  A scheduler thread owns the GPU work:
//   - admission: requests wait in arrival order until their device copies fit
//     under the memory budget; an admitted request is uploaded and put in
//     spatial order on an upload stream, overlapping the counting;
//   - skipping: once a request is in spatial order, the tile pairs of its
//     counts that lie wholly beyond the top edge are dropped (their pairs are
//     overflow), so rounds carry only tile pairs that can land in a bin;
//   - rounds: one persistent pair-count launch over a segment table drawn from
//     every admitted, ready request: small requests first (up to half of a
//     round), then the others in arrival order; a request that arrives while
//     others are counting joins the next round instead of queueing behind them
//     (rounds double while the backlog is deep); two rounds are in flight on
//     two streams, so that the next round's CTAs fill the SMs that the
//     current round's last CTAs leave idle;
//   - completion: after the round that holds a request's last tile pairs, the
//     overflow slots and the copy of its counts to the host are queued on the
//     same stream, so its counts are final when its event fires; w(theta) is
//     then evaluated on the host.
// There is no device-side wait on host data: every round is an ordinary
// launch.  Host waits (wtheta_server_wait) are bounded by the caller's timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "wtheta_internal.h"

namespace {

using namespace wtheta;
using Clock = std::chrono::steady_clock;

enum ReqState { kQueued = 0, kUploading = 1, kCounting = 2, kFinishing = 3, kDone = 4, kFailed = 5 };

struct Request {
    uint64_t id = 0;
    int kind = 0;                      // WTHETA_REQ_AUTO or WTHETA_REQ_CROSS
    int ncat = 0;                      // 2 or 4
    int ncount = 0;                    // 3 or 4
    long long n[4] = {0, 0, 0, 0};
    double* host_in[4] = {nullptr, nullptr, nullptr, nullptr};  // pinned copies
    size_t dev_bytes = 0;
    void* dmem = nullptr;
    Prepared prep[4];
    unsigned long long* d_counts = nullptr;      // ncount x (K+2)
    Segment* d_segs = nullptr;                   // the request's counts, for finalize
    Segment seg[4];                              // templates (item_offset = 0)
    long long sched[4] = {0, 0, 0, 0};           // tile pairs handed to rounds so far
    unsigned long long* host_counts = nullptr;   // pinned, ncount x (K+2), then 4 kept counts
    unsigned long long* d_kept = nullptr;        // tile pairs kept per count (far ones skipped)
    unsigned* d_list[4] = {nullptr, nullptr, nullptr, nullptr};  // kept items per count
    cudaEvent_t ready = nullptr, finished = nullptr;
    int state = kQueued;
    int status = WTHETA_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<double> w;
    long long pairs = 0;
    int cull = 0;                                // far tile pairs skipped
};

struct Round {
    cudaStream_t st = nullptr;     // its own stream: the next round's CTAs start as this
                                   // round's retire, so launch tails overlap
    Segment* d_segs = nullptr;
    Segment* h_segs = nullptr;     // pinned staging of the table
    int cap = 0;
    unsigned long long* d_cursor = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
};

}  // namespace

struct wtheta_server {
    int dev = 0;
    int K = 0;
    BinTable tab;
    const Variant* v = nullptr;
    size_t smem = 0;
    int grid = 0;
    int span = 1;              // settle (A group, B chunk) spans without a lookup per pair
    int cull = 1;              // skip tile pairs wholly beyond the top edge
    double theta_top = 0.0;    // top edge, radians
    int sm_count = 0;
    size_t budget = 0;
    size_t resident = 0;
    long long round_items = 0;
    int max_active = 0;
    cudaStream_t up = nullptr;
    Round rounds[2];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::map<uint64_t, Request*> all;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    Clock::time_point t0;
    // statistics
    long long n_rounds = 0, n_done = 0, items_done = 0, kernels = 0;
    double busy_s = 0;
};

namespace {

double now_s(const wtheta_server* S) {
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

// Tile pairs of count k of a request (catalogue pairs as in admit).
long long count_items(const Request* r, long long T, int k) {
    static const int auto_a[3] = {0, 0, 1}, auto_b[3] = {0, 1, 1};
    static const int cross_a[4] = {0, 0, 1, 1}, cross_b[4] = {2, 3, 2, 3};
    const bool aut = r->kind == WTHETA_REQ_AUTO;
    const long long ta = round_up(r->n[aut ? auto_a[k] : cross_a[k]], T) / T;
    const long long tb = round_up(r->n[aut ? auto_b[k] : cross_b[k]], T) / T;
    return aut && auto_a[k] == auto_b[k] ? ta * (ta + 1) / 2 : ta * tb;
}

size_t cull_bytes(const wtheta_server* S, const Request* r) {
    if (!r->cull) return 0;
    const long long T = (long long)S->v->nt * S->v->r;
    size_t b = 256;                                    // kept counters
    for (int c = 0; c + 1 < r->ncat; c += 2)           // caps of each prepared pair
        b += ((size_t)(round_up(r->n[c], T) / T + round_up(r->n[c + 1], T) / T) * sizeof(TileCap) +
              255) / 256 * 256;
    for (int k = 0; k < r->ncount; ++k) b += ((size_t)count_items(r, T, k) * 4 + 255) / 256 * 256;
    return b;
}

size_t request_bytes(const wtheta_server* S, const Request* r) {
    const long long T = (long long)S->v->nt * S->v->r;
    size_t b = 0;
    for (int c = 0; c + 1 < r->ncat; c += 2)
        b += (prepare_joint_bytes(r->n[c], round_up(r->n[c], T), r->n[c + 1],
                                  round_up(r->n[c + 1], T)) + 255) / 256 * 256;
    b += (size_t)r->ncount * (S->K + 2) * 8 + 256;    // counts
    b += sizeof(Segment) * 4 + 256;                    // the request's segment table
    b += cull_bytes(S, r);                             // caps and kept tile pairs
    return b;
}

void free_host(Request* r) {
    for (int c = 0; c < 4; ++c)
        if (r->host_in[c]) {
            cudaFreeHost(r->host_in[c]);
            r->host_in[c] = nullptr;
        }
    if (r->host_counts) {
        cudaFreeHost(r->host_counts);
        r->host_counts = nullptr;
    }
    if (r->ready) cudaEventDestroy(r->ready);
    if (r->finished) cudaEventDestroy(r->finished);
    r->ready = r->finished = nullptr;
}

// Admission: device memory from the stream-ordered pool on the upload
// stream, copies in, conversion and spatial ordering, counts zeroed.
int admit(wtheta_server* S, Request* r) {
    TraceRange trace("server_admit");
    const long long T = (long long)S->v->nt * S->v->r;
    int rc = dev_malloc_async(&r->dmem, r->dev_bytes, S->up);
    if (rc) return rc;
    unsigned char* p = (unsigned char*)r->dmem;
    r->d_counts = (unsigned long long*)p;
    p += ((size_t)r->ncount * (S->K + 2) * 8 + 255) / 256 * 256;
    r->d_segs = (Segment*)p;
    p += (sizeof(Segment) * 4 + 255) / 256 * 256;
    // The catalogues are prepared two by two, (D, R) of an auto request and
    // (D1, R1), (D2, R2) of a cross one, each pair by one pipeline (sentinel
    // tags 0-1 and 2-3, so that no count pairs two coinciding sentinels).
    for (int c = 0; c + 1 < r->ncat && !rc; c += 2) {
        const long long na = r->n[c], nb = r->n[c + 1];
        const long long pa = round_up(na, T), pb = round_up(nb, T);
        const size_t bytes = (prepare_joint_bytes(na, pa, nb, pb) + 255) / 256 * 256;
        // The raw RA/Dec of both (16 B/pt) is uploaded into the start of the
        // region, where the FP32 copies (16 B/pt, tile-padded) will go: the
        // conversion reads it before, in stream order, the gather overwrites it.
        unsigned char* region = p;
        p += bytes;
        rc = check_cuda(cudaMemcpyAsync(region, r->host_in[c], (size_t)na * 16,
                                        cudaMemcpyHostToDevice, S->up));
        if (!rc)
            rc = check_cuda(cudaMemcpyAsync(region + (size_t)na * 16, r->host_in[c + 1],
                                            (size_t)nb * 16, cudaMemcpyHostToDevice, S->up));
        if (rc) break;
        rc = prepare_joint((const double*)region, na, pa, (const double*)(region + (size_t)na * 16),
                           nb, pb, 0, c, region, S->sm_count, S->up, &r->prep[c],
                           &r->prep[c + 1]);
    }
    if (!rc) rc = check_cuda(cudaMemsetAsync(r->d_counts, 0, (size_t)r->ncount * (S->K + 2) * 8, S->up));
    if (rc) return rc;
    // the counts of the request
    auto tiles = [&](int c) { return round_up(r->n[c], T) / T; };
    auto pairs_of = [&](int a, int b, bool aut) -> unsigned long long {
        return aut ? (unsigned long long)r->n[a] * (unsigned long long)(r->n[a] - 1) / 2
                   : (unsigned long long)r->n[a] * (unsigned long long)r->n[b];
    };
    const int K2 = S->K + 2;
    if (r->kind == WTHETA_REQ_AUTO) {
        r->seg[0] = make_segment(r->prep[0], r->prep[0], tiles(0), tiles(0), 1, 0, r->d_counts, pairs_of(0, 0, true));
        r->seg[1] = make_segment(r->prep[0], r->prep[1], tiles(0), tiles(1), 0, 0, r->d_counts + K2, pairs_of(0, 1, false));
        r->seg[2] = make_segment(r->prep[1], r->prep[1], tiles(1), tiles(1), 1, 0, r->d_counts + 2 * K2, pairs_of(1, 1, true));
    } else {
        // catalogues: 0 = D1, 1 = R1, 2 = D2, 3 = R2; counts D1D2, D1R2, R1D2, R1R2
        r->seg[0] = make_segment(r->prep[0], r->prep[2], tiles(0), tiles(2), 0, 0, r->d_counts, pairs_of(0, 2, false));
        r->seg[1] = make_segment(r->prep[0], r->prep[3], tiles(0), tiles(3), 0, 0, r->d_counts + K2, pairs_of(0, 3, false));
        r->seg[2] = make_segment(r->prep[1], r->prep[2], tiles(1), tiles(2), 0, 0, r->d_counts + 2 * K2, pairs_of(1, 2, false));
        r->seg[3] = make_segment(r->prep[1], r->prep[3], tiles(1), tiles(3), 0, 0, r->d_counts + 3 * K2, pairs_of(1, 3, false));
    }
    r->pairs = 0;
    for (int k = 0; k < r->ncount; ++k) r->pairs += (long long)r->seg[k].total;
    rc = check_cuda(cudaMemcpyAsync(r->d_segs, r->seg, sizeof(Segment) * r->ncount,
                                    cudaMemcpyHostToDevice, S->up));
    if (!rc && r->cull) {
        // bounding caps of every catalogue's tiles, then each count's tile
        // pairs that may hold a pair below the top edge; the kept numbers come
        // back to the host before the request is ready
        r->d_kept = (unsigned long long*)p;
        p += 256;
        TileCap* caps[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int c = 0; c + 1 < r->ncat && !rc; c += 2) {
            // one launch over a prepared pair: the second's tiles follow the first's
            const long long ta = round_up(r->n[c], T) / T, tb = round_up(r->n[c + 1], T) / T;
            caps[c] = (TileCap*)p;
            caps[c + 1] = caps[c] + ta;
            p += ((size_t)(ta + tb) * sizeof(TileCap) + 255) / 256 * 256;
            if (ta + tb > 0)
                rc = launch_tile_caps(r->prep[c].p32, (ta + tb) * T, (int)T, ta + tb, caps[c],
                                      S->up);
        }
        if (!rc) rc = check_cuda(cudaMemsetAsync(r->d_kept, 0, 4 * 8, S->up));
        static const int auto_a[3] = {0, 0, 1}, auto_b[3] = {0, 1, 1};
        static const int cross_a[4] = {0, 0, 1, 1}, cross_b[4] = {2, 3, 2, 3};
        const bool aut = r->kind == WTHETA_REQ_AUTO;
        for (int k = 0; k < r->ncount && !rc; ++k) {
            r->d_list[k] = (unsigned*)p;
            p += ((size_t)r->seg[k].n_items * 4 + 255) / 256 * 256;
            const int a = aut ? auto_a[k] : cross_a[k], b = aut ? auto_b[k] : cross_b[k];
            rc = launch_cull_items(caps[a], caps[b], r->seg[k].tiles_a, r->seg[k].tiles_b,
                                   r->seg[k].is_auto, r->seg[k].n_items, S->theta_top,
                                   r->d_list[k], r->d_kept + k, S->sm_count, S->up);
        }
        if (!rc)
            rc = check_cuda(cudaMemcpyAsync(r->host_counts + (size_t)r->ncount * K2, r->d_kept,
                                            (size_t)r->ncount * 8, cudaMemcpyDeviceToHost, S->up));
    }
    if (!rc) rc = check_cuda(cudaEventRecord(r->ready, S->up));
    return rc;
}

// The request's uploads, ordering and skipping have finished: its counts
// take only the kept tile pairs.
void on_ready(const wtheta_server* S, Request* r) {
    if (!r->cull) return;
    const unsigned long long* kept = r->host_counts + (size_t)r->ncount * (S->K + 2);
    for (int k = 0; k < r->ncount; ++k) {
        r->seg[k].n_items = (long long)kept[k];
        r->seg[k].item_list = r->d_list[k];
    }
}

long long remaining(const Request* r) {
    long long x = 0;
    for (int k = 0; k < r->ncount; ++k) x += r->seg[k].n_items - r->sched[k];
    return x;
}

// Builds and launches one round on its stream; returns true if it launched
// one.  Called with the server lock held.
bool launch_round(wtheta_server* S, Round& R) {
    TraceRange trace("server_round");
    std::vector<Request*> ready;
    for (Request* r : S->active)
        if (r->state == kCounting && remaining(r) > 0) {
            ready.push_back(r);
        } else if (r->state == kUploading && cudaEventQuery(r->ready) == cudaSuccess) {
            r->state = kCounting;
            on_ready(S, r);
            ready.push_back(r);  // even with no tile pair left: it still has to finish
        }
    if (ready.empty()) return false;
    // Small requests (all their remaining tile pairs fit in an eighth of a
    // round) go first, up to half of the round, so that they are not held
    // behind large ones; the rest of the round goes to the others in arrival
    // order, each taking what it needs, so that a large request is delayed
    // only by earlier ones and by small ones.
    // With a deep backlog, rounds twice as long: fewer launch tails; a
    // request arriving meanwhile waits at most one such round.
    long long backlog = 0;
    for (Request* r : ready) backlog += remaining(r);
    long long budget = backlog > 16 * S->round_items ? 2 * S->round_items : S->round_items;
    const long long small_items = S->round_items / 8;
    long long small_budget = budget / 2;
    std::vector<long long> give(ready.size(), 0);
    for (size_t i = 0; i < ready.size() && small_budget > 0; ++i) {
        const long long rem = remaining(ready[i]);
        if (rem > small_items) continue;
        give[i] = std::min(rem, small_budget);
        small_budget -= give[i];
        budget -= give[i];
    }
    for (size_t i = 0; i < ready.size() && budget > 0; ++i) {
        const long long g = std::min(remaining(ready[i]) - give[i], budget);
        give[i] += g;
        budget -= g;
    }
    // segment table of the round
    int n = 0;
    long long items = 0;
    std::vector<Request*> finishing;
    for (size_t i = 0; i < ready.size() && n < R.cap; ++i) {
        Request* r = ready[i];
        long long g = give[i];
        for (int k = 0; k < r->ncount && g > 0 && n < R.cap; ++k) {
            const long long left = r->seg[k].n_items - r->sched[k];
            if (left <= 0) continue;
            const long long take = std::min(left, g);
            Segment sg = r->seg[k];
            sg.item_begin = items;
            sg.n_items = take;
            sg.item_offset = r->sched[k];
            R.h_segs[n++] = sg;
            r->sched[k] += take;
            items += take;
            g -= take;
        }
        if (remaining(r) == 0) finishing.push_back(r);
    }
    if (n == 0 && finishing.empty()) return false;
    // every request in the round must be ready on the round's stream
    for (Request* r : ready) cudaStreamWaitEvent(R.st, r->ready, 0);
    int rc = WTHETA_OK;
    if (n > 0) {
        rc = check_cuda(cudaMemcpyAsync(R.d_segs, R.h_segs, sizeof(Segment) * n,
                                        cudaMemcpyHostToDevice, R.st));
        if (!rc) rc = check_cuda(cudaMemsetAsync(R.d_cursor, 0, 8, R.st));
        const int grid = (int)std::min<long long>(S->grid, items);
        PairParams prm = make_params(S->v, S->tab, nullptr, R.d_segs, n, 0, items, R.d_cursor,
                                     nullptr);
        prm.span = S->span;
        if (!rc) rc = launch_pairs(S->v, prm, grid, S->smem, R.st);
        ++S->kernels;
    }
    // requests whose last tile pairs are in this round: overflow slots, then
    // their counts to the host, in stream order after the round and after the
    // other round in flight (which may hold earlier tile pairs of theirs)
    if (!finishing.empty())
        for (Round& O : S->rounds)
            if (&O != &R && O.busy) cudaStreamWaitEvent(R.st, O.done, 0);
    for (Request* r : finishing) {
        if (!rc) rc = launch_finalize_segments(r->d_segs, r->ncount, S->K, R.st);
        ++S->kernels;
        if (!rc)
            rc = check_cuda(cudaMemcpyAsync(r->host_counts, r->d_counts,
                                            (size_t)r->ncount * (S->K + 2) * 8,
                                            cudaMemcpyDeviceToHost, R.st));
        if (!rc) rc = check_cuda(cudaFreeAsync(r->dmem, R.st));
        if (!rc) r->dmem = nullptr;
        if (!rc) rc = check_cuda(cudaEventRecord(r->finished, R.st));
        r->state = rc ? kFailed : kFinishing;
        r->status = rc;
    }
    if (!rc) rc = check_cuda(cudaEventRecord(R.done, R.st));
    R.busy = !rc;
    ++S->n_rounds;
    S->items_done += items;
    return !rc;
}

void finish_request(wtheta_server* S, Request* r) {
    r->t_done = now_s(S);
    r->state = kDone;
    S->resident -= r->dev_bytes;
    r->w.assign(S->K, 0.0);
    const uint64_t* c = (const uint64_t*)r->host_counts;
    const int K2 = S->K + 2;
    if (r->kind == WTHETA_REQ_AUTO)
        r->status = wtheta_ls(c, c + K2, c + 2 * K2, r->n[0], r->n[1], S->K, r->w.data());
    else
        r->status = wtheta_ls_cross(c, c + K2, c + 2 * K2, c + 3 * K2, r->n[0], r->n[2], r->n[1],
                                    r->n[3], S->K, r->w.data());
    ++S->n_done;
}

void worker_loop(wtheta_server* S) {
    cudaSetDevice(S->dev);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progressed = false;
        // admission, in arrival order, while the budget allows
        while (!S->queue.empty() && (int)S->active.size() < S->max_active) {
            Request* r = S->queue.front();
            if (S->resident + r->dev_bytes > S->budget) break;
            S->queue.pop_front();
            r->t_admit = now_s(S);
            const int rc = admit(S, r);
            if (rc) {
                if (r->dmem) {
                    cudaFreeAsync(r->dmem, S->up);
                    r->dmem = nullptr;
                }
                r->state = kFailed;
                r->status = rc;
                r->t_done = now_s(S);
                S->cv_done.notify_all();
                continue;
            }
            S->resident += r->dev_bytes;
            r->state = kUploading;
            S->active.push_back(r);
            progressed = true;
        }
        // finished rounds free their slot
        for (Round& R : S->rounds)
            if (R.busy && cudaEventQuery(R.done) == cudaSuccess) {
                R.busy = false;
                progressed = true;
            }
        // completed requests
        for (size_t i = 0; i < S->active.size();) {
            Request* r = S->active[i];
            if ((r->state == kFinishing && cudaEventQuery(r->finished) == cudaSuccess) ||
                r->state == kFailed) {
                if (r->state == kFinishing) finish_request(S, r);
                else r->t_done = now_s(S);
                S->active.erase(S->active.begin() + i);
                S->cv_done.notify_all();
                progressed = true;
            } else {
                ++i;
            }
        }
        // keep two rounds in flight
        for (Round& R : S->rounds)
            if (!R.busy && launch_round(S, R)) progressed = true;
        if (!progressed) S->cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
}

int server_create(const double* edges, int K, size_t budget, int max_active,
                  const wtheta_tune* tune, wtheta_server** out) {
    if (!out || budget == 0 || max_active < 0) return WTHETA_EINVAL;
    wtheta_server* S = new wtheta_server();
    int rc = build_table(edges, K, &S->tab);
    DeviceInfo di;
    if (!rc) rc = device_info(&di);
    if (!rc) rc = check_cuda(cudaGetDevice(&S->dev));
    if (!rc) {
        S->K = K;
        S->budget = budget;
        S->max_active = max_active ? max_active : 1024;
        S->sm_count = di.sm_count;
        S->v = pick_variant(tune, K, S->tab.n_lut, di.max_smem_optin);
        S->span = !(tune && tune->span_bins == 2);
        S->cull = !(tune && tune->skip_far == 2) && edges[K] < 180.0;
        S->theta_top = edges[K] * (3.14159265358979323846 / 180.0);
        if (!S->v) rc = WTHETA_EINVAL;
    }
    if (!rc) {
        S->smem = S->v->smem(K, S->tab.n_lut);
        rc = grid_for(S->v, S->smem, 1LL << 40, di.sm_count, 0, &S->grid);
        // a round of ~48 tile pairs per CTA (about 10 ms of work): short
        // enough for new requests to join soon, long enough that the tail of
        // each launch stays small
        S->round_items = 48LL * S->grid;
    }
    // the upload stream runs at the highest priority: its short preparation
    // kernels take the SM slots that a round's last CTAs free before the CTAs
    // of the round waiting behind it, so a new request does not wait for whole
    // rounds to become ready
    int prio_low = 0, prio_high = 0;
    if (!rc) rc = check_cuda(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    if (!rc)
        rc = check_cuda(cudaStreamCreateWithPriority(&S->up, cudaStreamNonBlocking, prio_high));
    for (Round& R : S->rounds) {
        if (rc) break;
        R.cap = 4096;
        rc = check_cuda(cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking));
        if (!rc) rc = dev_malloc((void**)&R.d_segs, sizeof(Segment) * R.cap);
        if (!rc) rc = check_cuda(cudaMallocHost(&R.h_segs, sizeof(Segment) * R.cap));
        if (!rc) rc = dev_malloc((void**)&R.d_cursor, 8);
        if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming));
    }
    if (rc) {
        delete S;
        return rc;
    }
    S->t0 = Clock::now();
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return WTHETA_OK;
}

}  // namespace

extern "C" {

int wtheta_server_create(const double* bin_edges_deg, int32_t n_bins, size_t hbm_budget_bytes,
                         int32_t max_active, const wtheta_tune* tune, wtheta_server** server) {
    return server_create(bin_edges_deg, n_bins, hbm_budget_bytes, max_active, tune, server);
}

int wtheta_server_submit(wtheta_server* S, const wtheta_request* q, uint64_t* req_id) {
    if (!S || !q || !req_id) return WTHETA_EINVAL;
    if (q->kind != WTHETA_REQ_AUTO && q->kind != WTHETA_REQ_CROSS) return WTHETA_EINVAL;
    Request* r = new Request();
    r->kind = q->kind;
    r->ncat = q->kind == WTHETA_REQ_AUTO ? 2 : 4;
    r->ncount = q->kind == WTHETA_REQ_AUTO ? 3 : 4;
    const double* src[4] = {q->data, q->rand, q->data2, q->rand2};
    const long long n[4] = {q->n_data, q->n_rand, q->n_data2, q->n_rand2};
    int rc = WTHETA_OK;
    for (int c = 0; c < r->ncat; ++c)
        if (!src[c] || n[c] < 2) rc = WTHETA_EINVAL;
    if (!rc) {
        for (int c = 0; c < r->ncat; ++c) r->n[c] = n[c];
        // far tile pairs are skipped unless a count has 2^32 tile pairs or more
        // (kept items are listed by 32-bit index)
        const long long T = (long long)S->v->nt * S->v->r;
        r->cull = S->cull;
        for (int k = 0; k < r->ncount; ++k)
            if (count_items(r, T, k) >= (1LL << 32)) r->cull = 0;
        r->dev_bytes = request_bytes(S, r);
        if (r->dev_bytes > S->budget) rc = WTHETA_EBUDGET;
    }
    // the server keeps its own pinned copies of the inputs
    for (int c = 0; c < r->ncat && !rc; ++c) {
        rc = check_cuda(cudaMallocHost(&r->host_in[c], (size_t)n[c] * 16));
        if (!rc) std::memcpy(r->host_in[c], src[c], (size_t)n[c] * 16);
    }
    if (!rc) rc = check_cuda(cudaMallocHost(&r->host_counts, ((size_t)r->ncount * (S->K + 2) + 4) * 8));
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming));
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&r->finished, cudaEventDisableTiming));
    if (rc) {
        free_host(r);
        delete r;
        return rc;
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        r->id = S->next_id++;
        r->t_submit = now_s(S);
        S->all[r->id] = r;
        S->queue.push_back(r);
    }
    S->cv_work.notify_one();
    *req_id = r->id;
    return WTHETA_OK;
}

int wtheta_server_wait(wtheta_server* S, uint64_t id, int64_t timeout_ms, int32_t* done,
                       uint64_t* counts, double* w) {
    if (!S || !done) return WTHETA_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return WTHETA_EINVAL;
    Request* r = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max<int64_t>(timeout_ms, 0));
    while (r->state != kDone && r->state != kFailed) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            r->state != kDone && r->state != kFailed) {
            *done = 0;
            return timeout_ms > 0 ? WTHETA_ETIMEOUT : WTHETA_OK;
        }
    }
    *done = 1;
    if (r->state == kFailed) return r->status ? r->status : WTHETA_ECUDA;
    if (counts) std::memcpy(counts, r->host_counts, (size_t)r->ncount * (S->K + 2) * 8);
    if (w) std::memcpy(w, r->w.data(), sizeof(double) * S->K);
    return r->status;
}

int wtheta_server_request_info(wtheta_server* S, uint64_t id, wtheta_request_info* info) {
    if (!S || !info) return WTHETA_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return WTHETA_EINVAL;
    const Request* r = it->second;
    info->state = r->state;
    info->status = r->status;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_done = r->t_done;
    info->pairs = r->pairs;
    info->n_counts = r->ncount;
    return WTHETA_OK;
}

int wtheta_server_cancel(wtheta_server* S, uint64_t id) {
    if (!S) return WTHETA_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return WTHETA_EINVAL;
    Request* r = it->second;
    if (r->state != kQueued) return WTHETA_EBUSY;  // admitted: its work is on the device
    auto q = std::find(S->queue.begin(), S->queue.end(), r);
    if (q != S->queue.end()) S->queue.erase(q);
    r->state = kFailed;
    r->status = WTHETA_ECANCELED;
    r->t_done = now_s(S);
    S->cv_done.notify_all();
    S->cv_work.notify_all();
    return WTHETA_OK;
}

int wtheta_server_release(wtheta_server* S, uint64_t id) {
    if (!S) return WTHETA_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return WTHETA_EINVAL;
    Request* r = it->second;
    if (r->state != kDone && r->state != kFailed) return WTHETA_EINVAL;
    free_host(r);
    delete r;
    S->all.erase(it);
    return WTHETA_OK;
}

int wtheta_server_stats(wtheta_server* S, wtheta_server_stats_t* st) {
    if (!S || !st) return WTHETA_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    st->rounds = S->n_rounds;
    st->completed = S->n_done;
    st->queued = (int64_t)S->queue.size();
    st->active = (int64_t)S->active.size();
    st->items = S->items_done;
    st->resident_bytes = (int64_t)S->resident;
    st->kernels = S->kernels;
    return WTHETA_OK;
}

int wtheta_server_destroy(wtheta_server* S) {
    if (!S) return WTHETA_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->dev);
    for (Round& R : S->rounds)
        if (R.st) cudaStreamSynchronize(R.st);
    if (S->up) cudaStreamSynchronize(S->up);
    for (auto& kv : S->all) {
        Request* r = kv.second;
        if (r->dmem) cudaFree(r->dmem);
        free_host(r);
        delete r;
    }
    for (Round& R : S->rounds) {
        if (R.d_segs) cudaFree(R.d_segs);
        if (R.h_segs) cudaFreeHost(R.h_segs);
        if (R.d_cursor) cudaFree(R.d_cursor);
        if (R.done) cudaEventDestroy(R.done);
        if (R.st) cudaStreamDestroy(R.st);
    }
    if (S->up) cudaStreamDestroy(S->up);
    delete S;
    return WTHETA_OK;
}

}  // extern "C"
