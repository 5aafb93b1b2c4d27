// Serving loop: continuous batching of subdivision requests on one GPU.
//
// Requests arrive from any thread (alsub_serve_submit copies their host inputs) and wait in a FIFO.
// Worker threads, each owning some slots (a slot is a CUDA stream with an event and page-locked
// staging buffers), admit the head of the queue as soon as one of their slots is free and the
// request's device bytes fit the HBM budget, and retire slots whose event has completed, so
// requests overlap on the device and a new one joins as soon as another leaves. Two kinds:
//   FRAME  new control positions for a resident topology (Sec. 3.6 "Static topology": build once,
//          evaluate per frame): H2D, then one SpMV with the cached composite operator (Sec. 3.6
//          "Single SpMV evaluation") or the eval kernels on the cached topology, as chosen at
//          registration (optionally by a timed trial of both); D2H.
//   MESH   a new control mesh (Sec. 3.6 "Dynamic topology"): mesh upload, fused build + eval of
//          every level (alsub_subdivide), D2H; its handles are freed when the slot retires.
// Per-request device buffers come from the stream-ordered allocator on the slot's stream, so
// nothing in the loop synchronises the device. Every wait is bounded.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

using namespace alsub;

namespace {

constexpr size_t kMaxQueued = 1 << 16;

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t mesh_bytes(long long F, long long nnz, long long K) {
    return 4 * (size_t)(F + 1) + 4 * (size_t)nnz + 12 * (size_t)K;
}


struct Resident {
    alsub_mesh_t mesh = nullptr;
    alsub_topology_t topo = nullptr;
    alsub_operator_t op = nullptr;   // the composite (or matrix-free) operator frames run on
    int64_t V0 = 0, VL = 0;
    size_t bytes = 0;                // topology + mesh + operator + frame buffers
    // The frames' device buffers, the resident's own: with the same input and output every frame,
    // a repeated frame replays the topology's captured graph. Frames of the resident therefore run
    // one after another on the device: a frame's input copy waits for in_free (the previous frame's
    // kernels have read d_in) and its kernels for out_free (the previous output copy has read d_out).
    float *d_in = nullptr, *d_out = nullptr;
    cudaEvent_t in_free = nullptr, out_free = nullptr;
    // the topology's launch state (its graph cache, the fork and join events of its side streams)
    // and the two events are shared by every frame of this resident: one worker enqueues at a time
    std::mutex launch;
};

struct Job {
    uint64_t ticket = 0;
    int kind = 0;
    Resident *res = nullptr;
    alsub_scheme scheme = ALSUB_CATMULL_CLARK;
    int levels = 0;
    int V = 0, F = 0, K = 0, B = 0;   // B: boundary edges the request states (MESH)
    std::vector<int32_t> off, fv, cv;
    std::vector<float> cs, P0;
    int64_t VL = 0;
    size_t need = 0;                 // admission bytes while in flight
    float *user_out = nullptr;       // caller's output buffer (or null)
    bool user_pinned = false;
    double t_submit = 0, t_start = 0, t_done = 0;
    double host_start = 0, host_finish = 0;   // worker time spent enqueueing / retiring (s)
    alsub_status status = ALSUB_OK;
    bool done = false;
    bool by_operator = false;
    std::vector<float> out;          // result kept by the server when user_out is null
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_b = nullptr, ev_c = nullptr;  // timed: the request's compute begins / ends
    Job *job = nullptr;
    float *h_in = nullptr, *h_out = nullptr;   // page-locked staging
    size_t cap_in = 0, cap_out = 0;
    void *d_buf = nullptr;                     // this request's device buffers (one allocation)
    alsub_mesh_t mesh = nullptr;
    alsub_topology_t topo = nullptr;
};

bool grow_host(float **p, size_t *cap, size_t n) {
    if (*cap >= n && *p) return true;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMallocHost((void **)p, std::max<size_t>(n, 1) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    *cap = n;
    return true;
}

}  // namespace

struct alsub_server_s {
    size_t budget = 0, used = 0, peak = 0, resident_bytes = 0;
    std::vector<Slot> slots;
    std::vector<std::unique_ptr<Resident>> residents;   // never moved once made
    std::deque<Job *> queue;
    std::map<uint64_t, Job *> jobs;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    int running = 0;                 // requests admitted and not yet retired (all workers)
    int running_peak = 0;            // largest `running` seen
    cudaEvent_t t0 = nullptr;        // timed reference event, recorded at creation
    std::vector<std::pair<float, float>> dev_iv;   // completed requests' compute intervals (ms
                                                   // after t0, from the slot's events)
    bool stop = false, paused = false;
    int device = 0;
    cudaStream_t reg_stream = nullptr;
    cudaMemPool_t pool = nullptr;
    uint64_t old_threshold = 0;
    std::vector<double> lat;         // latencies of completed requests (s)
    double host_start_sum = 0, host_finish_sum = 0;
    double host_start_frames = 0, host_start_meshes = 0;   // host_start_sum split by kind
    int64_t completed = 0, failed = 0, frames_op = 0, frames_eval = 0, meshes = 0;
    double first_submit = -1, last_done = 0;
};

namespace {

// Enqueue one request on its slot. Runs on the worker thread, lock not held.
alsub_status start(Slot &sl, Job &j) {
    const size_t n_in = 3 * (size_t)j.V, n_out = 3 * (size_t)j.VL;
    const bool direct = j.user_out && j.user_pinned;    // D2H straight into the caller's buffer
    if (!grow_host(&sl.h_in, &sl.cap_in, n_in) || (!direct && !grow_host(&sl.h_out, &sl.cap_out, n_out)))
        return report(ALSUB_ERR_OOM, "server: page-locked staging allocation failed");
    memcpy(sl.h_in, j.P0.data(), 4 * n_in);
    float *dst = direct ? j.user_out : sl.h_out;
    if (j.kind == ALSUB_REQ_FRAME) {
        // the resident's own buffers, so a repeated frame replays one captured graph
        Resident *R = j.res;
        j.by_operator = R->op != nullptr;
        std::lock_guard<std::mutex> g(R->launch);
        cudaStreamWaitEvent(sl.stream, R->in_free, 0);
        if (cudaMemcpyAsync(R->d_in, sl.h_in, 4 * n_in, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return report(ALSUB_ERR_DEVICE, "server: input copy failed");
        cudaStreamWaitEvent(sl.stream, R->out_free, 0);
        cudaEventRecord(sl.ev_b, sl.stream);
        const alsub_status fs = R->op ? alsub_apply_operator(R->op, R->d_in, R->d_out, sl.stream)
                                      : alsub_refine_vertices(R->topo, R->d_in, R->d_out, nullptr, sl.stream);
        if (fs != ALSUB_OK) return fs;
        cudaEventRecord(R->in_free, sl.stream);
        cudaEventRecord(sl.ev_c, sl.stream);
        if (cudaMemcpyAsync(dst, R->d_out, 4 * n_out, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
            cudaEventRecord(R->out_free, sl.stream) != cudaSuccess ||
            cudaEventRecord(sl.ev, sl.stream) != cudaSuccess)
            return report(ALSUB_ERR_DEVICE, "server: output copy failed");
        return ALSUB_OK;
    }
    alsub_status st = ALSUB_OK;
    {
        // the stated boundary edge count is checked on the device (a different one is reported in
        // the request's status when it is retired): nothing here waits for the device
        const long long B = j.B;
        st = alsub::create_mesh(j.scheme, j.V, j.F, j.off.empty() ? nullptr : j.off.data(), j.fv.data(), j.K,
                                j.K ? j.cv.data() : nullptr, j.K ? j.cs.data() : nullptr, nullptr, &B, sl.stream,
                                &sl.mesh);
        if (st == ALSUB_OK) st = alsub_topology_create(sl.mesh, j.levels, sl.stream, &sl.topo);
        if (st != ALSUB_OK) return st;
    }
    const size_t b_in = align256(4 * n_in), b_out = align256(4 * n_out);
    if (cudaMallocAsync(&sl.d_buf, b_in + b_out, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        sl.d_buf = nullptr;
        return report(ALSUB_ERR_OOM, "server: device allocation failed");
    }
    float *d_in = (float *)sl.d_buf;
    float *d_out = (float *)((char *)sl.d_buf + b_in);
    if (cudaMemcpyAsync(d_in, sl.h_in, 4 * n_in, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return report(ALSUB_ERR_DEVICE, "server: input copy failed");
    cudaEventRecord(sl.ev_b, sl.stream);
    st = alsub_subdivide(sl.topo, d_in, d_out, nullptr, sl.stream);
    if (st != ALSUB_OK) return st;
    cudaEventRecord(sl.ev_c, sl.stream);
    if (cudaMemcpyAsync(dst, d_out, 4 * n_out, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaEventRecord(sl.ev, sl.stream) != cudaSuccess)
        return report(ALSUB_ERR_DEVICE, "server: output copy failed");
    return ALSUB_OK;
}

// Retire a slot whose work has completed (or failed to enqueue). Worker thread, lock not held.
void finish(alsub_server_s &S, Slot &sl, alsub_status st) {
    Job &j = *sl.job;
    const double h0 = now_s();
    if (st == ALSUB_OK && sl.topo) st = alsub_topology_status(sl.topo);  // latched device checks
    if (st == ALSUB_OK) {
        const size_t n_out = 3 * (size_t)j.VL;
        if (!j.user_out) j.out.assign(sl.h_out, sl.h_out + n_out);
        else if (!j.user_pinned) memcpy(j.user_out, sl.h_out, 4 * n_out);
    }
    float tb = -1.f, tc = -1.f;
    if (st == ALSUB_OK && (cudaEventElapsedTime(&tb, S.t0, sl.ev_b) != cudaSuccess ||
                           cudaEventElapsedTime(&tc, S.t0, sl.ev_c) != cudaSuccess))
        tb = tc = -1.f;
    if (sl.d_buf) cudaFreeAsync(sl.d_buf, sl.stream);
    sl.d_buf = nullptr;
    if (sl.topo) alsub_topology_destroy(sl.topo);
    if (sl.mesh) alsub_mesh_destroy(sl.mesh);
    sl.topo = nullptr;
    sl.mesh = nullptr;
    cudaGetLastError();
    const double t = now_s();
    j.host_finish = t - h0;
    std::lock_guard<std::mutex> g(S.mu);
    j.status = st;
    j.t_done = t;
    j.done = true;
    S.used -= j.need;
    S.running--;
    if (st == ALSUB_OK) {
        S.lat.push_back(t - j.t_submit);
        S.host_start_sum += j.host_start;
        (j.kind == ALSUB_REQ_MESH ? S.host_start_meshes : S.host_start_frames) += j.host_start;
        S.host_finish_sum += j.host_finish;
        S.completed++;
        S.last_done = t;
        if (tb >= 0.f) S.dev_iv.emplace_back(tb, tc);
        if (j.kind == ALSUB_REQ_MESH) S.meshes++;
        else if (j.by_operator) S.frames_op++;
        else S.frames_eval++;
    } else {
        S.failed++;
    }
    sl.job = nullptr;
    S.cv_done.notify_all();
}

// One worker owns slots [first, first + count): it retires them and admits into them.
void worker_loop(alsub_server_s *Sp, int first, int count) {
    alsub_server_s &S = *Sp;
    cudaSetDevice(S.device);
    Slot *mine = S.slots.data() + first;
    while (true) {
        bool progress = false;
        for (int i = 0; i < count; i++) {
            Slot &sl = mine[i];
            if (!sl.job) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            alsub_status st = ALSUB_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                st = report(ALSUB_ERR_DEVICE, cudaGetErrorString(q));
            }
            finish(S, sl, st);
            progress = true;
        }
        while (true) {
            Slot *free_slot = nullptr;
            bool busy = false;
            for (int i = 0; i < count; i++) {
                if (!mine[i].job && !free_slot) free_slot = &mine[i];
                busy |= mine[i].job != nullptr;
            }
            Job *j = nullptr;
            bool over = false;
            {
                std::lock_guard<std::mutex> g(S.mu);
                if (S.stop) return;
                if (!free_slot || S.paused || S.queue.empty()) break;
                Job *h = S.queue.front();
                if (S.used + h->need > S.budget) {
                    if (S.running > 0) break;  // wait for requests in flight to free memory
                    over = true;               // nothing in flight anywhere: it can never fit
                }
                S.queue.pop_front();
                if (over) {
                    h->need = 0;
                } else {
                    S.used += h->need;
                    S.peak = std::max(S.peak, S.used);
                }
                S.running++;
                S.running_peak = std::max(S.running_peak, S.running);
                j = h;
            }
            progress = true;
            busy = true;
            j->t_start = now_s();
            free_slot->job = j;
            if (over) {
                finish(S, *free_slot, report(ALSUB_ERR_OOM, "server: request does not fit the budget"));
                continue;
            }
            const alsub_status st = start(*free_slot, *j);
            j->host_start = now_s() - j->t_start;
            if (st != ALSUB_OK) {
                cudaStreamSynchronize(free_slot->stream);
                finish(S, *free_slot, st);
            }
        }
        if (progress) continue;
        bool busy = false;
        for (int i = 0; i < count; i++) busy |= mine[i].job != nullptr;
        std::unique_lock<std::mutex> lk(S.mu);
        if (S.stop) return;
        // in flight: look at the events again after 20 us; idle: sleep until a submit (or 5 ms)
        S.cv_work.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::microseconds(5000));
    }
}

void free_resident(Resident &R) {
    if (R.in_free) cudaEventSynchronize(R.in_free);
    if (R.out_free) cudaEventSynchronize(R.out_free);
    if (R.d_in) cudaFree(R.d_in);
    if (R.d_out) cudaFree(R.d_out);
    if (R.in_free) cudaEventDestroy(R.in_free);
    if (R.out_free) cudaEventDestroy(R.out_free);
    R.d_in = R.d_out = nullptr;
    R.in_free = R.out_free = nullptr;
    if (R.op) alsub_operator_destroy(R.op);
    if (R.topo) alsub_topology_destroy(R.topo);
    if (R.mesh) alsub_mesh_destroy(R.mesh);
    R.op = nullptr;
    R.topo = nullptr;
    R.mesh = nullptr;
}

// Mean time of `reps` runs of fn() on stream s (after one warm-up run), CUDA events.
template <class Fn>
float time_ms(cudaStream_t s, int reps, Fn fn) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) { cudaGetLastError(); return 1e30f; }
    if (cudaEventCreate(&b) != cudaSuccess) { cudaGetLastError(); cudaEventDestroy(a); return 1e30f; }
    fn();
    cudaEventRecord(a, s);
    for (int i = 0; i < reps; i++) fn();
    cudaEventRecord(b, s);
    float ms = 1e30f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) ms /= reps;
    else ms = 1e30f;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGetLastError();
    return ms;
}

}  // namespace

extern "C" {

alsub_status alsub_serve_create(size_t budget, int32_t max_slots, alsub_server_t *out) {
    if (!out || max_slots <= 0 || max_slots > 64 || budget == 0)
        return report(ALSUB_ERR_INVALID_ARG, "server: max_slots must be 1..64 and the budget > 0");
    *out = nullptr;
    std::unique_ptr<alsub_server_s> S(new (std::nothrow) alsub_server_s());
    if (!S) return report(ALSUB_ERR_OOM, "host allocation failed");
    S->budget = budget;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        return report(ALSUB_ERR_DEVICE, "no CUDA device");
    }
    S->slots.resize(max_slots);
    bool ok = cudaStreamCreateWithFlags(&S->reg_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (Slot &sl : S->slots)
        ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&sl.ev_b) == cudaSuccess && cudaEventCreate(&sl.ev_c) == cudaSuccess;
    ok = ok && cudaEventCreate(&S->t0) == cudaSuccess && cudaEventRecord(S->t0, S->reg_stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (S->t0) cudaEventDestroy(S->t0);
        for (Slot &sl : S->slots) {
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.ev_b) cudaEventDestroy(sl.ev_b);
            if (sl.ev_c) cudaEventDestroy(sl.ev_c);
            if (sl.stream) cudaStreamDestroy(sl.stream);
        }
        if (S->reg_stream) cudaStreamDestroy(S->reg_stream);
        return report(ALSUB_ERR_DEVICE, "server: stream creation failed");
    }
    if (cudaDeviceGetDefaultMemPool(&S->pool, S->device) == cudaSuccess &&
        cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &S->old_threshold) == cudaSuccess) {
        uint64_t th = std::max<uint64_t>(S->old_threshold, budget);
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &th);
    } else {
        S->pool = nullptr;
    }
    cudaGetLastError();
    // one worker thread per two slots (at most 8): the host side of a request (validation,
    // allocation, launches) takes long enough that one thread would cap the request rate.
    // ALSUB_SERVE_WORKERS overrides the count (1 .. max_slots).
    int nw = std::max(1, std::min(8, max_slots / 2));
    if (const char *env = getenv("ALSUB_SERVE_WORKERS")) {
        const int w = atoi(env);
        if (w >= 1) nw = std::min(w, max_slots);
    }
    for (int w = 0, first = 0; w < nw; w++) {
        const int count = max_slots / nw + (w < max_slots % nw ? 1 : 0);
        S->workers.emplace_back(worker_loop, S.get(), first, count);
        first += count;
    }
    *out = S.release();
    return ALSUB_OK;
}

alsub_status alsub_serve_register(alsub_server_t S, alsub_scheme scheme, int32_t V, int32_t F,
                                  const int32_t *off, const int32_t *fv, int32_t K, const int32_t *cv,
                                  const float *cs, int32_t levels, int32_t frame_path, int32_t *resident) {
    if (!S || !resident || frame_path < ALSUB_FRAMES_EVAL ||
        frame_path > ALSUB_FRAMES_OPERATOR_MATRIX_FREE)
        return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    cudaSetDevice(S->device);
    cudaStream_t s = S->reg_stream;
    std::unique_ptr<Resident> R(new (std::nothrow) Resident());
    if (!R) return report(ALSUB_ERR_OOM, "host allocation failed");
    alsub_status st = alsub_mesh_create(scheme, V, F, off, fv, K, cv, cs, s, &R->mesh);
    if (st != ALSUB_OK) return st;
    {
        // closed-form size first: a topology that cannot fit is never built
        float smax = 0.f;
        for (int i = 0; i < K; i++) smax = std::max(smax, cs[i]);
        const int32_t nnz = off ? off[F] : F * (scheme == ALSUB_CATMULL_CLARK ? 4 : 3);
        size_t tb = 0;
        int64_t B = 0;
        alsub_mesh_boundary_edges(R->mesh, &B);
        st = alsub_plan_bytes(scheme, V, F, nnz, (int32_t)B, K, smax, levels, &tb);
        std::lock_guard<std::mutex> g(S->mu);
        if (st == ALSUB_OK && S->used + tb > S->budget)
            st = report(ALSUB_ERR_OOM, "server: the resident topology does not fit the budget");
    }
    const TopoImpl *P = nullptr;
    if (st == ALSUB_OK) st = alsub_refine_topology(R->mesh, levels, s, &R->topo);
    if (st == ALSUB_OK) st = alsub_topology_status(R->topo);
    if (st != ALSUB_OK) {
        cudaStreamSynchronize(s);
        free_resident(*R);
        return st;
    }
    P = topology_impl(R->topo);
    const size_t mb = mesh_bytes(P->mesh->F, P->mesh->nnz, P->mesh->K);
    R->V0 = V;
    R->VL = P->L[levels].V;
    size_t tbytes = 0;
    alsub_topology_bytes(R->topo, &tbytes);
    R->bytes = tbytes + mb;
    if (frame_path == ALSUB_FRAMES_OPERATOR_MATRIX_FREE && levels > 0) {
        // the stencil kernels on the cached topology behind alsub_apply_operator: no matrix, only
        // the operator's own scratch (the intermediate levels)
        alsub_operator_t op = nullptr;
        st = alsub_build_operator(R->topo, ALSUB_OP_MATRIX_FREE, s, &op);
        if (st != ALSUB_OK) {
            cudaStreamSynchronize(s);
            free_resident(*R);
            return st;
        }
        size_t ob = 0;
        alsub_operator_bytes(op, &ob);
        R->op = op;
        R->bytes = tbytes + mb + ob;
    } else if (frame_path != ALSUB_FRAMES_EVAL && levels > 0) {
        alsub_operator_t op = nullptr;
        if (alsub_build_operator(R->topo, ALSUB_OP_COMPOSE, s, &op) == ALSUB_OK) {
            size_t ob = 0;
            alsub_operator_bytes(op, &ob);
            alsub_topology_bytes(R->topo, &tbytes);   // the build may have stored more per-corner arrays
            bool fits;
            {
                std::lock_guard<std::mutex> g(S->mu);
                fits = S->used + tbytes + mb + ob <= S->budget;
            }
            float t_op = 0.f, t_eval = 1.f;   // OPERATOR: keep R whenever it fits
            if (fits && frame_path == ALSUB_FRAMES_FASTEST) {
                t_op = 1e30f;
                t_eval = 0.f;
                // trial: frames by each path on zero positions (the values do not change the time)
                void *buf = nullptr;
                const size_t n0 = align256(12 * (size_t)R->V0), nl = align256(12 * (size_t)R->VL);
                if (cudaMallocAsync(&buf, n0 + nl, s) == cudaSuccess) {
                    cudaMemsetAsync(buf, 0, n0, s);
                    const float *p0 = (const float *)buf;
                    float *pl = (float *)((char *)buf + n0);
                    t_op = time_ms(s, 3, [&] { alsub_apply_operator(op, p0, pl, s); });
                    t_eval = time_ms(s, 3, [&] { alsub_refine_vertices(R->topo, p0, pl, nullptr, s); });
                    cudaFreeAsync(buf, s);
                }
                cudaGetLastError();
            }
            if (fits && t_op < t_eval) {
                R->op = op;
                R->bytes = tbytes + mb + ob;
            } else {
                alsub_operator_destroy(op);
                R->bytes = tbytes + mb;
            }
        }
        cudaGetLastError();
    }
    {
        // the frames' buffers and the events that order the frames on the device
        const size_t io = align256(12 * (size_t)R->V0) + align256(12 * (size_t)R->VL);
        bool ok = cudaMalloc(&R->d_in, align256(12 * (size_t)R->V0)) == cudaSuccess &&
                  cudaMalloc(&R->d_out, align256(12 * (size_t)R->VL)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            cudaStreamSynchronize(s);
            free_resident(*R);
            return report(ALSUB_ERR_OOM, "server: frame buffer allocation failed");
        }
        ok = cudaEventCreateWithFlags(&R->in_free, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&R->out_free, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            cudaStreamSynchronize(s);
            free_resident(*R);
            return report(ALSUB_ERR_DEVICE, "server: event creation failed");
        }
        R->bytes += io;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        free_resident(*R);
        return report(ALSUB_ERR_DEVICE, "server: registration failed");
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->used + R->bytes > S->budget) {
        free_resident(*R);
        return report(ALSUB_ERR_OOM, "server: the resident topology does not fit the budget");
    }
    S->used += R->bytes;
    S->resident_bytes += R->bytes;
    S->peak = std::max(S->peak, S->used);
    S->residents.push_back(std::move(R));
    *resident = (int32_t)S->residents.size() - 1;
    return ALSUB_OK;
}

alsub_status alsub_serve_submit(alsub_server_t S, const alsub_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket || !r->P0_host) return report(ALSUB_ERR_INVALID_ARG, "bad request");
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return report(ALSUB_ERR_OOM, "host allocation failed");
    j->kind = r->kind;
    j->user_out = r->PL_host;
    if (r->kind == ALSUB_REQ_FRAME) {
        std::lock_guard<std::mutex> g(S->mu);
        if (r->resident < 0 || r->resident >= (int)S->residents.size())
            return report(ALSUB_ERR_INVALID_ARG, "unknown resident topology");
        Resident *R = S->residents[r->resident].get();
        j->res = R;
        j->V = (int)R->V0;
        j->VL = R->VL;
        j->need = 0;                 // a frame runs in its resident's buffers
    } else if (r->kind == ALSUB_REQ_MESH) {
        if (r->num_verts <= 0 || r->num_faces <= 0 || !r->face_verts_host || r->levels < 0 ||
            r->scheme < ALSUB_CATMULL_CLARK || r->scheme > ALSUB_SQRT3 || r->num_creases < 0 ||
            (r->num_creases > 0 && (!r->crease_verts_host || !r->crease_sharpness_host)))
            return report(ALSUB_ERR_INVALID_ARG, "bad mesh request");
        j->scheme = (alsub_scheme)r->scheme;
        j->levels = r->levels;
        j->V = r->num_verts;
        j->F = r->num_faces;
        const long long order = r->scheme == ALSUB_CATMULL_CLARK ? 4 : 3;
        j->off.resize((size_t)j->F + 1);
        if (r->face_offsets_host) {
            memcpy(j->off.data(), r->face_offsets_host, 4 * ((size_t)j->F + 1));
            if (j->off[0] != 0) return report(ALSUB_ERR_INVALID_ARG, "face_offsets[0] must be 0");
            for (int f = 0; f < j->F; f++)
                if (j->off[f + 1] < j->off[f]) return report(ALSUB_ERR_INVALID_ARG, "face offsets decrease");
        } else {
            if (order * j->F > 0x7fffffffLL) return report(ALSUB_ERR_UNSUPPORTED, "counts exceed int32");
            for (int f = 0; f <= j->F; f++) j->off[f] = (int32_t)(f * order);
        }
        const int nnz = j->off[j->F];
        j->fv.assign(r->face_verts_host, r->face_verts_host + nnz);
        j->K = r->num_creases;
        float smax = 0.f;
        if (j->K > 0) {
            j->cv.assign(r->crease_verts_host, r->crease_verts_host + 2 * (size_t)j->K);
            j->cs.assign(r->crease_sharpness_host, r->crease_sharpness_host + j->K);
            for (float x : j->cs)
                if (x > smax) smax = x;   // NaN or negative values are refused when the request runs
        }
        size_t tb = 0;
        j->B = r->num_boundary_edges;
        alsub_status st = alsub_plan_bytes(j->scheme, j->V, j->F, nnz, j->B, j->K, smax, j->levels, &tb);
        if (st != ALSUB_OK) return st;
        std::vector<int64_t> c(4 * ((size_t)j->levels + 1));
        alsub_plan_open(j->scheme, j->V, j->F, nnz, j->B, j->levels, c.data());
        j->VL = c[4 * (size_t)j->levels];
        j->need = tb + mesh_bytes(j->F, nnz, j->K) + align256(12 * (size_t)j->V) + align256(12 * (size_t)j->VL);
    } else {
        return report(ALSUB_ERR_INVALID_ARG, "unknown request kind");
    }
    if (j->user_out) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, j->user_out) == cudaSuccess) {
            if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
                return report(ALSUB_ERR_INVALID_ARG, "PL_host must be host memory");
            j->user_pinned = a.type == cudaMemoryTypeHost;
        }
        cudaGetLastError();
    }
    j->P0.assign(r->P0_host, r->P0_host + 3 * (size_t)j->V);
    std::lock_guard<std::mutex> g(S->mu);
    if (S->resident_bytes + j->need > S->budget)
        return report(ALSUB_ERR_OOM, "server: the request is larger than the budget left by the residents");
    if (S->queue.size() >= kMaxQueued) return report(ALSUB_ERR_BUSY, "server: the queue is full");
    j->ticket = S->next_ticket++;
    j->t_submit = now_s();
    if (S->first_submit < 0) S->first_submit = j->t_submit;
    Job *jp = j.release();
    S->jobs[jp->ticket] = jp;
    S->queue.push_back(jp);
    *ticket = jp->ticket;
    S->cv_work.notify_all();
    return ALSUB_OK;
}

alsub_status alsub_serve_poll(alsub_server_t S, uint64_t ticket, int32_t timeout_us, alsub_result *res) {
    if (!S || !res || timeout_us < 0) return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return report(ALSUB_ERR_INVALID_ARG, "unknown ticket");
    Job *j = it->second;
    if (!j->done && timeout_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return j->done; });
    if (!j->done)
        return timeout_us > 0 ? report(ALSUB_ERR_TIMEOUT, "request still in flight")
                              : report(ALSUB_ERR_NOT_READY, "request still in flight");
    res->status = j->status;
    res->kind = j->kind;
    res->num_verts = j->VL;
    res->PL_host = j->status != ALSUB_OK ? nullptr : (j->user_out ? j->user_out : j->out.data());
    res->submit_s = j->t_submit;
    res->start_s = j->t_start;
    res->done_s = j->t_done;
    return ALSUB_OK;
}

alsub_status alsub_serve_release(alsub_server_t S, uint64_t ticket) {
    if (!S) return report(ALSUB_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end() || !it->second->done)
        return report(ALSUB_ERR_INVALID_ARG, "no finished request with this ticket");
    delete it->second;
    S->jobs.erase(it);
    return ALSUB_OK;
}

alsub_status alsub_serve_pause(alsub_server_t S, int32_t paused) {
    if (!S) return report(ALSUB_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    S->paused = paused != 0;
    S->cv_work.notify_all();
    return ALSUB_OK;
}

alsub_status alsub_serve_stats_get(alsub_server_t S, alsub_serve_stats *st) {
    if (!S || !st) return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    std::lock_guard<std::mutex> g(S->mu);
    std::vector<double> l = S->lat;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {   // nearest rank
        if (l.empty()) return 0.0;
        size_t k = (size_t)ceil(p * (double)l.size());
        return l[std::min(l.size(), std::max<size_t>(k, 1)) - 1];
    };
    memset(st, 0, sizeof(*st));
    st->completed = S->completed;
    st->failed = S->failed;
    st->queued = (int64_t)S->queue.size();
    for (const Slot &sl : S->slots) st->in_flight += sl.job != nullptr;
    st->p50_ms = 1e3 * pct(0.50);
    st->p99_ms = 1e3 * pct(0.99);
    double sum = 0;
    for (double x : l) sum += x;
    st->mean_ms = l.empty() ? 0 : 1e3 * sum / (double)l.size();
    st->max_ms = l.empty() ? 0 : 1e3 * l.back();
    const double span = S->last_done - S->first_submit;
    st->throughput_rps = (S->completed && span > 0) ? (double)S->completed / span : 0;
    st->hbm_budget = S->budget;
    st->hbm_in_use = S->used;
    st->hbm_peak = S->peak;
    st->frames_operator = S->frames_op;
    st->frames_eval = S->frames_eval;
    st->meshes = S->meshes;
    st->host_start_ms_mean = S->completed ? 1e3 * S->host_start_sum / (double)S->completed : 0;
    st->host_finish_ms_mean = S->completed ? 1e3 * S->host_finish_sum / (double)S->completed : 0;
    const int64_t nf = S->frames_op + S->frames_eval;
    st->host_start_frame_ms_mean = nf ? 1e3 * S->host_start_frames / (double)nf : 0;
    st->host_start_mesh_ms_mean = S->meshes ? 1e3 * S->host_start_meshes / (double)S->meshes : 0;
    st->peak_in_flight = S->running_peak;
    // most compute intervals open at one instant (an interval's end sorts before a start at the
    // same time, so touching intervals do not count as overlapping)
    std::vector<std::pair<float, int>> ev;
    ev.reserve(2 * S->dev_iv.size());
    for (const auto &iv : S->dev_iv) {
        ev.emplace_back(iv.first, 1);
        ev.emplace_back(iv.second, -1);
    }
    std::sort(ev.begin(), ev.end());
    int64_t open = 0;
    for (const auto &e : ev) st->device_overlap_peak = std::max(st->device_overlap_peak, open += e.second);
    return ALSUB_OK;
}

alsub_status alsub_serve_destroy(alsub_server_t S) {
    if (!S) return ALSUB_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->paused = true;
    }
    // let the requests in flight finish (bounded: 60 s), then stop the worker
    const double t0 = now_s();
    while (now_s() - t0 < 60.0) {
        bool busy = false;
        {
            std::lock_guard<std::mutex> g(S->mu);
            for (const Slot &sl : S->slots) busy |= sl.job != nullptr;
        }
        if (!busy) break;
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(S->device);
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.d_buf) cudaFreeAsync(sl.d_buf, sl.stream);
        if (sl.topo) alsub_topology_destroy(sl.topo);
        if (sl.mesh) alsub_mesh_destroy(sl.mesh);
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.ev_b) cudaEventDestroy(sl.ev_b);
        if (sl.ev_c) cudaEventDestroy(sl.ev_c);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (S->t0) cudaEventDestroy(S->t0);
    for (auto &R : S->residents) free_resident(*R);
    if (S->reg_stream) {
        cudaStreamSynchronize(S->reg_stream);
        cudaStreamDestroy(S->reg_stream);
    }
    if (S->pool) cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &S->old_threshold);
    for (auto &kv : S->jobs) delete kv.second;   // queued requests are in `jobs` too
    cudaGetLastError();
    delete S;
    return ALSUB_OK;
}

}  // extern "C"
