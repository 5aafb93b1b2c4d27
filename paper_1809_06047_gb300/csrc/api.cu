// C ABI of libalsub: host validation, handles, closed-form allocation and the per-level
// orchestration of the build (topology) and eval (vertex) steps.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace alsub;

struct alsub_mesh_s {
    MeshImpl m;
};
struct alsub_topology_s {
    TopoImpl t;
};

namespace {

thread_local std::string g_err;

alsub_status fail(alsub_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

alsub_status cuda_fail(cudaError_t e, const char *what) {
    return fail(ALSUB_ERR_DEVICE, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            if (e_ == cudaErrorMemoryAllocation) {                                 \
                cudaGetLastError();                                                \
                return fail(ALSUB_ERR_OOM, "%s: out of device memory", #call);     \
            }                                                                      \
            return cuda_fail(e_, #call);                                           \
        }                                                                          \
    } while (0)

const long long kI32 = 2147483647LL;

// Closed-form counts of one refinement step from level l (Sec. 3.1 step 4, Appendix A, B): o =
// V, F, nnz, E and B (boundary edges) of level l + 1. Catmull-Clark and Loop split every boundary
// edge in two. sqrt(3) with feature edges (Kobbelt 2000): the first step of a pair (l even) keeps
// them; the second (l odd) splits them in three, which adds one vertex and one edge per boundary
// edge beyond the triangle slots (with B = 0, E + 3F is the closed mesh's 9F / 2).
bool next_counts(alsub_scheme s, int l, long long V, long long F, long long nnz, long long E, long long B,
                 long long *o) {
    if (s == ALSUB_CATMULL_CLARK) { o[0] = V + F + E; o[1] = nnz; o[2] = 4 * nnz; o[3] = 2 * E + nnz; o[4] = 2 * B; }
    else if (s == ALSUB_LOOP) { o[0] = V + E; o[1] = 4 * F; o[2] = 12 * F; o[3] = 2 * E + 3 * F; o[4] = 2 * B; }
    else {
        const long long b = (l & 1) ? B : 0;
        o[0] = V + F + b; o[1] = 3 * F; o[2] = 9 * F; o[3] = E + 3 * F + b; o[4] = (l & 1) ? 3 * B : B;
    }
    for (int i = 0; i < 5; i++)
        if (o[i] > kI32) return false;
    return true;
}

// Device arrays of a handle: sizes rounded to 256 bytes; carved from the handle's arena while it
// has room (the arrays made at creation), else allocated one by one (arrays added later).
template <class T>
alsub_status dalloc(TopoImpl &T_, T **p, size_t n, cudaStream_t s) {
    *p = nullptr;
    if (n == 0) n = 1;
    const size_t b = (n * sizeof(T) + 255) & ~(size_t)255;
    T_.bytes += b;
    if (T_.dry) return ALSUB_OK;
    if (T_.arena && T_.arena_off + b <= T_.arena_size) {
        *p = (T *)(T_.arena + T_.arena_off);
        T_.arena_off += b;
        return ALSUB_OK;
    }
    void *q = nullptr;
    cudaError_t e = dev_malloc(T_.alloc, &q, n * sizeof(T), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ALSUB_ERR_OOM, "device allocation of %zu bytes failed", n * sizeof(T));
    }
    T_.allocs.push_back(q);
    *p = (T *)q;
    return ALSUB_OK;
}

#define AL(ptr, n)                                                   \
    do {                                                             \
        alsub_status st_ = dalloc(T, &(ptr), (size_t)(n), s);        \
        if (st_ != ALSUB_OK) return st_;                             \
    } while (0)

void free_topo(TopoImpl &T) {
    for (void *p : T.allocs) dev_free(T.alloc, p, T.stream);
    T.allocs.clear();
    T.bytes = 0;
    T.arena = nullptr;
    T.arena_off = T.arena_size = 0;
}

alsub_status alloc_crease(TopoImpl &T, CreaseList &C, long long cap, bool table, cudaStream_t s) {
    C.cap = cap;
    AL(C.count, 1);
    // a level without creases keeps count 0 for good (only the inheritance into a level with
    // capacity writes a count), so it is cleared here once instead of on every call
    if (cap == 0 && !T.dry) cudaMemsetAsync(C.count, 0, sizeof(int), s);
    if (cap > 0) {
        AL(C.edge, cap);
        AL(C.own, cap);
        AL(C.sig, cap);
        AL(C.verts, 2 * cap);
        AL(C.info, 2 * cap);
        if (table) {
            int k = 4;                                   // at least 16 slots, load factor <= 1/4
            while ((1LL << k) < 4 * cap) k++;
            C.hmask = (1 << k) - 1;
            C.hshift = 32 - k;
            AL(C.tab, (size_t)1 << k);
            AL(C.xverts, 2 * cap);
            AL(C.xsig, cap);
            AL(C.xcount, 1);
        }
    }
    return ALSUB_OK;
}

alsub_status topo_layout(TopoImpl &T, MeshImpl &M, int levels, cudaStream_t s);

// Sizes every array of the handle in a dry pass, makes one allocation of that size, and lays the
// arrays out in it (the same pass, for real).
alsub_status topo_alloc(TopoImpl &T, MeshImpl &M, int levels, cudaStream_t s) {
    if (T.dry) return topo_layout(T, M, levels, s);
    TopoImpl D;
    D.dry = true;
    alsub_status st = topo_layout(D, M, levels, s);
    if (st != ALSUB_OK) return st;
    void *q = nullptr;
    T.mesh = &M;
    T.alloc = M.alloc;
    if (dev_malloc(M.alloc, &q, D.bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(ALSUB_ERR_OOM, "device allocation of %zu bytes failed", D.bytes);
    }
    T.allocs.push_back(q);
    T.arena = (char *)q;
    T.arena_size = D.bytes;
    T.arena_off = 0;
    st = topo_layout(T, M, levels, s);
    T.arena_size = T.arena_off;                  // later arrays are allocated on their own
    return st;
}

alsub_status topo_layout(TopoImpl &T, MeshImpl &M, int levels, cudaStream_t s) {
    T.mesh = &M;
    T.alloc = M.alloc;
    T.scheme = M.scheme;
    T.levels = levels;
    T.stream = s;
    if (levels >= kMaxLevels) return fail(ALSUB_ERR_UNSUPPORTED, "at most %d levels", kMaxLevels - 1);
    T.L.assign(levels + 1, LevelBuf());
    LevelBuf &L0 = T.L[0];
    // every edge has two corners except the B boundary edges (one each)
    L0.V = M.V; L0.F = M.F; L0.nnz = M.nnz; L0.E = (M.nnz + M.B) / 2; L0.B = M.B;
    for (int l = 0; l < levels; l++) {
        long long o[5];
        LevelBuf &A = T.L[l];
        if (!next_counts(M.scheme, l, A.V, A.F, A.nnz, A.E, A.B, o))
            return fail(ALSUB_ERR_UNSUPPORTED, "level %d exceeds int32 counts", l + 1);
        LevelBuf &B = T.L[l + 1];
        B.V = o[0]; B.F = o[1]; B.nnz = o[2]; B.E = o[3]; B.B = o[4];
    }
    // sqrt(3) with feature edges takes the general path of sqrt3f.cu
    T.s3f = M.scheme == ALSUB_SQRT3 && (M.B > 0 || M.K > 0);
    const int V = M.V, nnz = M.nnz, E0 = (int)L0.E;
    L0.fv = M.d_fv;
    AL(L0.ce, nnz);
    AL(L0.tw, nnz);
    AL(T.cf0, nnz); AL(T.nx0, nnz); AL(T.pv0, nnz); AL(T.own0, nnz); AL(T.rn0, nnz); AL(T.eid, nnz);
    AL(T.vc0, V); AL(T.deg, V);
    if (M.scheme == ALSUB_CATMULL_CLARK) AL(T.rec0, (size_t)kRecInts * nnz);
    {
        int k = 4;                                   // directed-edge table: load factor <= 1/2
        while ((1LL << k) < 2LL * nnz) k++;
        T.dir.mask = (unsigned)((1LL << k) - 1);
        AL(T.dir.key, (size_t)1 << k);
        AL(T.dir.val, (size_t)1 << k);
    }
    AL(T.eo0, E0);
    AL(T.e0count, 1); AL(T.status, 1);
    // boundary lists of an open mesh, levels 0 .. levels - 1: the B_l = 2^l B boundary edges of
    // level l (each boundary edge splits into two, Sec. 3.2 "Boundaries")
    if (M.B > 0 && M.scheme != ALSUB_SQRT3) {
        AL(T.bcount, 1);
        for (int l = 0; l < levels; l++) {
            LevelBuf &A = T.L[l];
            AL(A.bA, A.B); AL(A.bE, A.B); AL(A.bS, A.B);
        }
    }
    // crease capacities: the sharpness of level l is at most sigma_max - l (each inherited
    // value is at most the parent maximum minus one), so creases are dead once l >= sigma_max
    bool creases = M.scheme != ALSUB_SQRT3 && M.K > 0;
    long long maxcap = 0;
    for (int l = 0; l <= levels; l++) {
        long long cap = 0;
        if (creases && (double)l < (double)M.sigma_max)
            cap = l == 0 ? M.K : std::min(2 * T.L[l - 1].cr.cap, T.L[l].E);
        alsub_status st = alloc_crease(T, T.L[l].cr, cap, true, s);
        if (st) return st;
        maxcap = std::max(maxcap, cap);
    }
    if (T.s3f) {
        // sqrt(3) feature path: every level's feature flags and twins, the export list of its
        // crease edges (K_l: the first step of a pair keeps them, the second splits them in three),
        // and the per-vertex scratch of the steps
        long long K = M.K, vmax3 = 1;
        for (int l = 0; l <= levels; l++) {
            LevelBuf &A = T.L[l];
            if (l < levels) {
                AL(A.fm, A.F);
                if (l > 0) AL(A.vc, A.V);
            }
            A.cr.cap = K;
            if (K > 0) {
                AL(A.cr.xverts, 2 * K);
                AL(A.cr.xsig, K);
                AL(A.cr.xcount, 1);
            }
            if (l < levels) vmax3 = std::max(vmax3, A.V);
            K = (l & 1) ? 3 * K : K;
        }
        AL(T.s3_vi, vmax3);
    }
    long long nflags = std::max<long long>({(long long)nnz, (long long)E0, 2 * maxcap, 1});
    AL(T.flags, nflags);
    AL(T.pos, nflags);
    T.scan_tmp_bytes = scan_tmp_bytes(std::max<long long>(nflags, V));
    AL(*(char **)&T.scan_tmp, T.scan_tmp_bytes);
    // Per-corner edge ids and twins are stored for every level that a later step reads them from.
    // Loop and sqrt(3) derive the last level's from its parent's. The last two Catmull-Clark steps
    // derive them instead: level levels - 1 (>= 2) from its
    // parent, and level levels - 2 (>= 2) from its parent too, the last step then going back two
    // levels; a level whose creases are still alive keeps them (its crease analysis walks rings
    // through them).
    T.L[0].helpers = true;
    for (int l = 1; l <= levels; l++) {
        LevelBuf &B = T.L[l];
        AL(B.fv, B.nnz);
        B.helpers = l < levels;
        const bool cc = M.scheme == ALSUB_CATMULL_CLARK;
        if (cc && l == levels - 1 && l >= 2 && B.cr.cap == 0) B.helpers = false;
        if (cc && l == levels - 2 && l >= 2 && B.cr.cap == 0 && T.L[levels - 1].cr.cap == 0)
            B.helpers = false;
        // Loop and sqrt(3): the last step derives its level's edge ids and twins from the parent
        // level (crease analysis included); its vertex rings are read from the parent level.
        if (!cc && l == levels - 1 && l >= 1) B.helpers = false;
        if (T.s3f) B.helpers = l < levels; // the general sqrt(3) path stores the twins below the last
        if (B.helpers) {
            if (M.scheme != ALSUB_SQRT3) AL(B.ce, B.nnz);
            AL(B.tw, B.nnz);
        }
    }
    long long vmax = 0;
    for (int l = 1; l < levels; l++) vmax = std::max(vmax, T.L[l].V);
    // two intermediate levels in flight, positions padded to float4 rows
    T.scratch_bytes = vmax > 0 ? 2 * 4 * sizeof(float) * (size_t)vmax : 0;
    if (T.scratch_bytes) AL(*(char **)&T.scratch, T.scratch_bytes);
    return ALSUB_OK;
}

void step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s) {
    if (T.scheme == ALSUB_CATMULL_CLARK) cc_step(T, l, topo, helpers, P, Pn, s);
    else if (T.scheme == ALSUB_LOOP) loop_step(T, l, topo, helpers, P, Pn, s);
    else sqrt3_step(T, l, topo, helpers, P, Pn, s);
}

// Ping-pong buffers of the intermediate levels.
void level_buffers(TopoImpl &T, const float *P0, float *PL, void *scratch, int l, const float **in,
                   float **out) {
    float *buf = scratch ? (float *)scratch : T.scratch;
    size_t half = T.scratch_bytes / (2 * sizeof(float));
    *in = l == 0 ? P0 : buf + half * ((l - 1) & 1);
    *out = l == T.levels - 1 ? PL : buf + half * (l & 1);
}

alsub_status finish(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return ALSUB_OK;
}

// Event k (0 .. levels + 1) of the current timed call, or nothing when timing is off. While a
// call is captured, slot 0's events stand in: the replay points the nodes at the call's slot.
void mark(TopoImpl &T, int k, cudaStream_t s) {
    if (!T.tcap) return;
    if (T.capturing) {
        cudaEventRecordWithFlags(T.tev[k], s, cudaEventRecordExternal);
        return;
    }
    const int slot = std::min(T.tcalls, T.tcap);
    cudaEventRecord(T.tev[(size_t)slot * (T.levels + 2) + k], s);
}

void drop_graph(CallGraph &G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = CallGraph();
}

void drop_graphs(TopoImpl &T) {
    for (auto &kind : T.graphs)
        for (CallGraph &G : kind) drop_graph(G);
}

void free_events(TopoImpl &T) {
    drop_graphs(T);                 // timed graphs hold these events
    for (cudaEvent_t e : T.tev) cudaEventDestroy(e);
    T.tev.clear();
    T.tcap = 0;
    T.tcalls = 0;
}

using Body = void (*)(TopoImpl &, const float *, float *, void *, cudaStream_t);
void ensure_side(TopoImpl &T);

// Run one refine call through a CUDA graph: captured (on a private stream) when a call repeats
// the previous call's pointers, replayed on `s` while they stay the same, so a repeated call costs
// one graph launch instead of one launch per kernel and memset. One-off calls and graphs that
// cannot be made launch the kernels directly, on `s` alone (the parallel crease branch of a
// subdivide call, with its stream and events, is made only for a graph). Calls on the handle's
// own buffers (own_buffers) are captured at once: they recur by construction.
alsub_status run_call(TopoImpl &T, int kind, const float *P0, float *PL, void *scratch, cudaStream_t s,
                      Body body, bool own_buffers = false) {
    const bool timed = T.tcap > 0;
    CallGraph *G = nullptr, *lru = &T.graphs[kind][0];
    for (CallGraph &g : T.graphs[kind]) {
        if (g.exec && g.P0 == P0 && g.PL == PL && g.scratch == scratch && g.timed == timed) G = &g;
        if (g.used < lru->used) lru = &g;
    }
    if (!G) {
        const void **prev = T.last[kind];
        const bool repeat = prev[0] == P0 && prev[1] == PL && prev[2] == scratch;
        prev[0] = P0; prev[1] = PL; prev[2] = scratch;
        if (!repeat && !own_buffers) {   // a one-off call: plain launches, no capture cost
            body(T, P0, PL, scratch, s);
            return finish("refine call");
        }
        G = lru;
        drop_graph(*G);
        ensure_side(T);      // the crease branch and the ring stream, for the graph of a repeated call
        bool ok = T.cap || cudaStreamCreateWithFlags(&T.cap, cudaStreamNonBlocking) == cudaSuccess;
        const long long before = T.launches;
        cudaGraph_t g = nullptr;
        if (ok) ok = cudaStreamBeginCapture(T.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            T.capturing = true;
            body(T, P0, PL, scratch, T.cap);
            T.capturing = false;
            ok = cudaStreamEndCapture(T.cap, &g) == cudaSuccess && g;
        }
        G->launches = T.launches - before;
        T.launches = before;
        if (ok && timed) {
            size_t n = 0;
            cudaGraphGetNodes(g, nullptr, &n);
            std::vector<cudaGraphNode_t> nodes(n);
            cudaGraphGetNodes(g, nodes.data(), &n);
            G->marks.assign(T.levels + 2, nullptr);
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType t;
                cudaEvent_t ev;
                if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
                if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
                for (int k = 0; k < T.levels + 2; k++)
                    if (ev == T.tev[k]) G->marks[k] = nd;
            }
            for (cudaGraphNode_t nd : G->marks) ok = ok && nd;
        }
        if (ok) ok = cudaGraphInstantiate(&G->exec, g, 0) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            *G = CallGraph();
            body(T, P0, PL, scratch, s);
            return finish("refine call");
        }
        G->graph = g;
        G->P0 = P0; G->PL = PL; G->scratch = scratch;
        G->timed = timed;
    }
    G->used = ++T.graph_clock;
    if (timed) {
        const size_t b = (size_t)std::min(T.tcalls, T.tcap) * (T.levels + 2);
        for (int k = 0; k < T.levels + 2; k++)
            CK(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->marks[k], T.tev[b + k]));
    }
    CK(cudaGraphLaunch(G->exec, s));
    T.launches += G->launches;
    return finish("refine call");
}

void refine_body(TopoImpl &T, const float *P0, float *PL, void *scratch, cudaStream_t s) {
    if (T.levels == 0) {
        cudaMemcpyAsync(PL, P0, sizeof(float) * 3 * (size_t)T.L[0].V, cudaMemcpyDeviceToDevice, s);
        return;
    }
    mark(T, 0, s);
    mark(T, 1, s);
    for (int l = 0; l < T.levels; l++) {
        const float *in;
        float *out;
        level_buffers(T, P0, PL, scratch, l, &in, &out);
        step(T, l, false, false, in, out, s);
        crease_fix(T, l, in, out, s);     // from the analysis kept at build time
        apply_edits(T, l + 1, out, s);
        mark(T, l + 2, s);
    }
}

void free_side(TopoImpl &T) {
    for (cudaEvent_t e : T.fork_ev) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : T.join_ev) if (e) cudaEventDestroy(e);
    T.fork_ev.clear();
    T.join_ev.clear();
    if (T.ring_ev) cudaEventDestroy(T.ring_ev);
    T.ring_ev = nullptr;
    if (T.rfork) cudaEventDestroy(T.rfork);
    if (T.rjoin) cudaEventDestroy(T.rjoin);
    if (T.rside) cudaStreamDestroy(T.rside);
    T.rfork = T.rjoin = nullptr;
    T.rside = nullptr;
    if (T.side) cudaStreamDestroy(T.side);
    T.side = nullptr;
}

// The side stream and fork / join events of alsub_subdivide (made before any capture). If any of
// them cannot be made, everything made is released and the call runs on the caller's stream alone.
void ensure_side(TopoImpl &T) {
    if (T.side) return;
    bool ok = cudaStreamCreateWithFlags(&T.side, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) T.side = nullptr;
    T.fork_ev.assign(T.levels + 1, nullptr);
    T.join_ev.assign(T.levels + 1, nullptr);
    for (int l = 0; ok && l <= T.levels; l++)
        ok = cudaEventCreateWithFlags(&T.fork_ev[l], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&T.join_ev[l], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&T.ring_ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok && T.scheme == ALSUB_CATMULL_CLARK)
        ok = cudaStreamCreateWithFlags(&T.rside, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&T.rfork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&T.rjoin, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_side(T);
    }
}


void free_hostio(TopoImpl &T) {
    TopoImpl::HostIO &io = T.io;
    if (io.cs) cudaStreamSynchronize(io.cs);
    if (io.ds) cudaStreamSynchronize(io.ds);
    for (int b = 0; b < 2; b++) {
        if (io.dPL[b]) dev_free(T.alloc, io.dPL[b], T.stream);
        if (io.hP0[b]) cudaFreeHost(io.hP0[b]);
        for (cudaEvent_t e : {io.up[b], io.done[b], io.copied[b]})
            if (e) cudaEventDestroy(e);
    }
    if (io.dP0) dev_free(T.alloc, io.dP0, T.stream);
    if (io.cs) cudaStreamDestroy(io.cs);
    if (io.ds) cudaStreamDestroy(io.ds);
    io = TopoImpl::HostIO();
    cudaGetLastError();
}

// Streams, events and buffers of alsub_subdivide_host, made at its first call (all or nothing).
alsub_status ensure_hostio(TopoImpl &T) {
    TopoImpl::HostIO &io = T.io;
    if (io.ready) return ALSUB_OK;
    const size_t n0 = 12 * (size_t)T.L[0].V, nl = 12 * (size_t)T.L[T.levels].V;
    bool ok = cudaStreamCreateWithFlags(&io.cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&io.ds, cudaStreamNonBlocking) == cudaSuccess &&
              dev_malloc(T.alloc, &io.dP0, n0, io.cs) == cudaSuccess;
    for (int b = 0; ok && b < 2; b++)
        ok = dev_malloc(T.alloc, &io.dPL[b], nl, io.cs) == cudaSuccess &&
             cudaMallocHost(&io.hP0[b], n0) == cudaSuccess &&
             cudaEventCreateWithFlags(&io.up[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&io.done[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&io.copied[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_hostio(T);
        return fail(ALSUB_ERR_OOM, "host-buffer subdivision: allocation failed");
    }
    io.ready = true;
    return ALSUB_OK;
}

// Dynamic topology. The crease analysis of level l needs level l's adjacency but no positions, so
// it runs on a side branch beside the build + eval of level l (forked when the step that built
// level l has been enqueued) and joins before the crease fix of level l:
//   main:  L0 build | step 0 | fix 0 | step 1 | fix 1 | ...
//   side:           L0 creases, analyse 0 | analyse 1 | ...
void subdivide_body(TopoImpl &T, const float *P0, float *PL, void *scratch, cudaStream_t s) {
    cudaStream_t z = T.side ? T.side : s;
    // analysis of level l on the side branch: it starts once everything enqueued on s so far (the
    // build of level l) is done, and its join event is recorded before anything else goes on z
    auto analyse_beside = [&](int l, bool level0) {
        if (z != s) {
            cudaEventRecord(T.fork_ev[l], s);
            cudaStreamWaitEvent(z, T.fork_ev[l], 0);
        }
        if (level0) level0_creases(T, z);
        crease_analyse(T, l, true, z);
        if (z != s) cudaEventRecord(T.join_ev[l], z);
    };
    auto wait_analysis = [&](int l) {
        if (z != s) cudaStreamWaitEvent(s, T.join_ev[l], 0);
    };
    mark(T, 0, s);
    level0_build(T, s);
    if (T.s3f) s3f_level0(T, s);
    // the side branch: the level-0 crease list and analysis, then the level-0 vertex checks (they
    // only set the status word, so nothing waits for them before the end of the call)
    if (crease_alive(T, 0)) {
        analyse_beside(0, true);
    } else {
        level0_creases(T, s);
        if (z != s) {
            cudaEventRecord(T.fork_ev[0], s);
            cudaStreamWaitEvent(z, T.fork_ev[0], 0);
        }
    }
    level0_validate(T, z);                  // also writes the ring records the steps >= 2 read
    if (z != s) cudaEventRecord(T.ring_ev, z);
    mark(T, 1, s);
    auto join_all = [&] {                   // everything on the side branch, before the call ends
        if (z == s) return;
        cudaEventRecord(T.join_ev[T.levels], z);
        cudaStreamWaitEvent(s, T.join_ev[T.levels], 0);
    };
    if (T.levels == 0) {
        join_all();
        cudaMemcpyAsync(PL, P0, sizeof(float) * 3 * (size_t)T.L[0].V, cudaMemcpyDeviceToDevice, s);
        return;
    }
    for (int l = 0; l < T.levels; l++) {
        const float *in;
        float *out;
        level_buffers(T, P0, PL, scratch, l, &in, &out);
        if (l == 2 && z != s) cudaStreamWaitEvent(s, T.ring_ev, 0);
        step(T, l, true, T.L[l + 1].helpers, in, out, s);
        if (l + 1 < T.levels && crease_alive(T, l + 1)) analyse_beside(l + 1, false);
        if (crease_alive(T, l)) {
            wait_analysis(l);
            crease_fix(T, l, in, out, s);
        }
        apply_edits(T, l + 1, out, s);
        if (l == T.levels - 1) join_all();
        mark(T, l + 2, s);
    }
}

}  // namespace

namespace alsub {
namespace {
__global__ void k_edit(int n, const int *__restrict__ vid, const float *__restrict__ off, int V, float *P, bool s4,
                       int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = vid[i];
    if (v < 0 || v >= V) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    const float3 d = f3(off[3 * i], off[3 * i + 1], off[3 * i + 2]);
    stpv(P, v, ldpv_rw(P, v, s4) + d, s4);
}

}  // namespace
}  // namespace alsub

// The edits of level k (1 .. levels) on its freshly refined positions `out`.
void alsub::apply_edits(TopoImpl &T, int k, float *out, cudaStream_t s) {
    if (k >= (int)T.edits.size() || T.edits[k].n == 0) return;
    const TopoImpl::LevelEdits &e = T.edits[k];
    k_edit<<<grid_for(e.n), kBlock, 0, s>>>(e.n, e.vid, e.off, (int)T.L[k].V, out, k < T.levels, T.status);
    T.launches += 1;
}

alsub_status alsub::report(alsub_status s, const char *msg) { return fail(s, "%s", msg); }

cudaError_t alsub::dev_malloc(const DevAlloc &A, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (A.alloc) {
        *p = A.alloc(bytes, A.ctx, (void *)s);
        // the arrays carved from an allocation need 16-byte alignment (vector and bulk accesses)
        if (*p && (reinterpret_cast<uintptr_t>(*p) & 15)) {
            A.free(*p, A.ctx, (void *)s);
            *p = nullptr;
        }
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
}

void alsub::dev_free(const DevAlloc &A, void *p, cudaStream_t s) {
    if (!p) return;
    if (A.free) A.free(p, A.ctx, (void *)s);
    else cudaFreeAsync(p, s);
}

alsub_status alsub::refine_call(TopoImpl &T, const float *P0, float *PL, void *scratch, cudaStream_t s) {
    if (!T.built) return fail(ALSUB_ERR_INVALID_ARG, "topology not built");
    alsub_status st = run_call(T, 0, P0, PL, scratch, s, refine_body);
    if (T.tcap && T.levels > 0) T.tcalls++;
    return st;
}

alsub_status alsub::refine_direct(TopoImpl &T, const float *P0, float *PL, void *scratch, cudaStream_t s) {
    if (!T.built) return fail(ALSUB_ERR_INVALID_ARG, "topology not built");
    refine_body(T, P0, PL, scratch, s);
    if (T.tcap && T.levels > 0) T.tcalls++;
    return finish("refine call");
}

TopoImpl *alsub::topology_impl(alsub_topology_t h) { return &h->t; }

alsub_status alsub::ensure_helpers(TopoImpl &T, cudaStream_t s) {
    bool changed = false;
    for (int l = 1; l < T.levels; l++) {
        LevelBuf &B = T.L[l];
        if (B.helpers) continue;
        if (T.scheme != ALSUB_SQRT3) AL(B.ce, B.nnz);
        AL(B.tw, B.nnz);
        B.helpers = true;
        changed = true;
        // redo the build of level l from level l - 1, now also emitting its edge ids and twins
        step(T, l - 1, true, true, nullptr, nullptr, s);
    }
    if (changed) drop_graphs(T);   // captured subdivide calls skipped those arrays
    return finish("ensure_helpers");
}

alsub_status alsub::create_mesh(alsub_scheme scheme, int32_t V, int32_t F, const int32_t *off_h,
                                const int32_t *fv_h, int32_t K, const int32_t *cv_h, const float *cs_h,
                                const alsub_allocator *allocator, const long long *B_stated, void *stream,
                                alsub_mesh_t *out) {
    if (!out) return fail(ALSUB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(ALSUB_ERR_INVALID_ARG, "allocator: both alloc and free are needed");
    *out = nullptr;
    if (scheme < ALSUB_CATMULL_CLARK || scheme > ALSUB_SQRT3) return fail(ALSUB_ERR_INVALID_ARG, "bad scheme");
    if (V <= 0 || F <= 0 || !fv_h || K < 0 || (K > 0 && (!cv_h || !cs_h)))
        return fail(ALSUB_ERR_INVALID_ARG, "bad mesh arguments");
    const int order = scheme == ALSUB_CATMULL_CLARK ? 4 : 3;
    std::vector<int32_t> off(F + 1);
    if (off_h) {
        if (off_h[0] != 0) return fail(ALSUB_ERR_INVALID_ARG, "face_offsets[0] must be 0");
        for (int r = 0; r < F; r++) {
            long long c = (long long)off_h[r + 1] - off_h[r];
            if (c < 3) return fail(ALSUB_ERR_INVALID_ARG, "face %d has order %lld < 3", r, c);
            if (scheme != ALSUB_CATMULL_CLARK && c != 3)
                return fail(ALSUB_ERR_INVALID_ARG, "face %d is not a triangle", r);
        }
        memcpy(off.data(), off_h, sizeof(int32_t) * (F + 1));
    } else {
        if ((long long)F * order > kI32) return fail(ALSUB_ERR_UNSUPPORTED, "counts exceed int32");
        for (int r = 0; r <= F; r++) off[r] = r * order;
    }
    const long long nnz = off[F];
    std::vector<int> used(V, 0), mark(V, -1);
    for (int r = 0; r < F; r++) {
        for (int x = off[r]; x < off[r + 1]; x++) {
            int v = fv_h[x];
            if (v < 0 || v >= V) return fail(ALSUB_ERR_INVALID_ARG, "face %d: vertex id %d out of range", r, v);
            if (mark[v] == r) return fail(ALSUB_ERR_INVALID_ARG, "face %d repeats vertex %d", r, v);
            mark[v] = r;
            used[v] = 1;
        }
    }
    for (int v = 0; v < V; v++)
        if (!used[v]) return fail(ALSUB_ERR_INVALID_ARG, "vertex %d is in no face", v);
    std::vector<int32_t> cv;
    std::vector<float> cs;
    float smax = 0.f;
    for (int i = 0; i < K; i++) {
        int a = cv_h[2 * i], b = cv_h[2 * i + 1];
        float sg = cs_h[i];
        if (a < 0 || a >= V || b < 0 || b >= V || a == b)
            return fail(ALSUB_ERR_INVALID_ARG, "crease %d: bad endpoints (%d, %d)", i, a, b);
        if (!(sg >= 0.f)) return fail(ALSUB_ERR_INVALID_ARG, "crease %d: sharpness must be >= 0", i);
        // sqrt(3) keeps the infinitely sharp creases (feature edges); finite sharpness has no
        // sqrt(3) rule
        if (sg == 0.f || (scheme == ALSUB_SQRT3 && !isinf(sg))) continue;
        cv.push_back(a); cv.push_back(b); cs.push_back(sg);
        smax = std::max(smax, sg);
    }
    alsub_mesh_s *h = new (std::nothrow) alsub_mesh_s();
    if (!h) return fail(ALSUB_ERR_OOM, "host allocation failed");
    MeshImpl &M = h->m;
    if (allocator) {
        M.alloc.alloc = allocator->alloc;
        M.alloc.free = allocator->free;
        M.alloc.ctx = allocator->ctx;
    }
    M.scheme = scheme; M.V = V; M.F = F; M.nnz = (int)nnz; M.K = (int)cs.size();
    M.sigma_max = smax;
    M.stream = (cudaStream_t)stream;
    cudaStream_t s = M.stream;
    upload_weight_tables();
    s3f_upload_tables();
    auto cleanup = [&]() {
        if (M.d_block) dev_free(M.alloc, M.d_block, s);
        delete h;
    };
    // one allocation: face offsets, corners, crease pairs and sharpness, the status word
    const size_t b_off = align256(sizeof(int) * ((size_t)F + 1)), b_fv = align256(sizeof(int) * (size_t)nnz);
    const size_t b_cv = align256(sizeof(int) * 2 * (size_t)M.K), b_cs = align256(sizeof(float) * (size_t)M.K);
    cudaError_t e = dev_malloc(M.alloc, &M.d_block, b_off + b_fv + b_cv + b_cs + 256, s);
    if (e == cudaSuccess) {
        char *p = (char *)M.d_block;
        M.d_off = (int *)p;
        M.d_fv = (int *)(p + b_off);
        M.d_cv = M.K ? (int *)(p + b_off + b_fv) : nullptr;
        M.d_cs = M.K ? (float *)(p + b_off + b_fv + b_cv) : nullptr;
        M.d_status = (int *)(p + b_off + b_fv + b_cv + b_cs);
        e = cudaMemsetAsync(M.d_status, 0, sizeof(int), s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.d_off, off.data(), sizeof(int) * (F + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.d_fv, fv_h, sizeof(int) * nnz, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && M.K) e = cudaMemcpyAsync(M.d_cv, cv.data(), sizeof(int) * 2 * M.K, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && M.K) e = cudaMemcpyAsync(M.d_cs, cs.data(), sizeof(float) * M.K, cudaMemcpyHostToDevice, s);
    // the host vectors (off, cv, cs) die on return: the copies complete at the stream
    // synchronisation below (the boundary scan's, which runs after them on the same stream)
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        cleanup();
        if (e == cudaErrorMemoryAllocation) return fail(ALSUB_ERR_OOM, "mesh upload: out of device memory");
        return cuda_fail(e, "mesh upload");
    }
    if (B_stated) {
        // the caller's count, checked on the device: a different one fails the builds that follow
        alsub_status st = mesh_boundary_check(M, s, *B_stated);
        if (st != ALSUB_OK) {
            cudaStreamSynchronize(s);          // the uploads read the host vectors
            cudaGetLastError();
            cleanup();
            return st;
        }
        // (copies from pageable host memory have been staged when cudaMemcpyAsync returns, so the
        // local vectors may die on return)
    } else {
        // boundary edges (Sec. 3.2 "Boundaries"; Loop takes the same rules, sqrt(3) Kobbelt's):
        // their number sizes every level; the paper gives no rule for a crease that meets the
        // boundary, so such input is refused
        long long B = 0;
        bool crease_at_boundary = false;
        alsub_status st = mesh_boundary_scan(M, s, &B, &crease_at_boundary);
        if (st == ALSUB_OK && crease_at_boundary)
            st = fail(ALSUB_ERR_UNSUPPORTED, "a crease touches a boundary vertex");
        if (st == ALSUB_OK && ((nnz + B) % 2 || B > kI32))
            st = fail(ALSUB_ERR_NONMANIFOLD, "inconsistent boundary (a directed edge repeats)");
        if (st != ALSUB_OK) {
            cudaStreamSynchronize(s);          // the uploads read the host vectors
            cudaGetLastError();
            cleanup();
            return st;
        }
        M.B = (int)B;
    }
    *out = h;
    return ALSUB_OK;
}

extern "C" {

const char *alsub_last_error(void) { return g_err.c_str(); }

const char *alsub_status_string(alsub_status s) {
    switch (s) {
        case ALSUB_OK: return "ALSUB_OK";
        case ALSUB_ERR_INVALID_ARG: return "ALSUB_ERR_INVALID_ARG";
        case ALSUB_ERR_NONMANIFOLD: return "ALSUB_ERR_NONMANIFOLD";
        case ALSUB_ERR_UNSUPPORTED: return "ALSUB_ERR_UNSUPPORTED";
        case ALSUB_ERR_OOM: return "ALSUB_ERR_OOM";
        case ALSUB_ERR_TIMEOUT: return "ALSUB_ERR_TIMEOUT";
        case ALSUB_ERR_DEVICE: return "ALSUB_ERR_DEVICE";
        case ALSUB_ERR_BUSY: return "ALSUB_ERR_BUSY";
        case ALSUB_ERR_NOT_READY: return "ALSUB_ERR_NOT_READY";
    }
    return "ALSUB_ERR_UNKNOWN";
}

alsub_status alsub_copy(void *dst, const void *src, size_t bytes, void *stream) {
    if (bytes == 0) return ALSUB_OK;
    if (!dst || !src) return fail(ALSUB_ERR_INVALID_ARG, "NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return ALSUB_OK;
}

alsub_status alsub_plan(alsub_scheme scheme, int64_t V, int64_t F, int64_t nnz, int32_t levels,
                        int64_t *counts) {
    return alsub_plan_open(scheme, V, F, nnz, 0, levels, counts);
}

alsub_status alsub_plan_open(alsub_scheme scheme, int64_t V, int64_t F, int64_t nnz, int64_t B,
                             int32_t levels, int64_t *counts) {
    if (scheme < ALSUB_CATMULL_CLARK || scheme > ALSUB_SQRT3) return fail(ALSUB_ERR_INVALID_ARG, "bad scheme");
    if (V <= 0 || F <= 0 || nnz < 3 * F || levels < 0 || !counts || B < 0 || B > nnz)
        return fail(ALSUB_ERR_INVALID_ARG, "bad counts");
    if (scheme != ALSUB_CATMULL_CLARK && nnz != 3 * F)
        return fail(ALSUB_ERR_INVALID_ARG, "Loop and sqrt(3) need a triangle mesh");
    if ((nnz + B) % 2) {
        if (B == 0) return fail(ALSUB_ERR_UNSUPPORTED, "odd corner count: the mesh is not closed");
        return fail(ALSUB_ERR_INVALID_ARG, "nnz + boundary edges must be even");
    }
    if (V > kI32 || F > kI32 || nnz > kI32) return fail(ALSUB_ERR_UNSUPPORTED, "counts exceed int32");
    long long c[5] = {V, F, nnz, (nnz + B) / 2, B};
    for (int l = 0; l <= levels; l++) {
        for (int i = 0; i < 4; i++) counts[4 * l + i] = c[i];
        if (l == levels) break;
        long long o[5];
        if (!next_counts(scheme, l, c[0], c[1], c[2], c[3], c[4], o))
            return fail(ALSUB_ERR_UNSUPPORTED, "level %d exceeds int32 counts", l + 1);
        memcpy(c, o, sizeof(c));
    }
    return ALSUB_OK;
}

alsub_status alsub_mesh_create(alsub_scheme scheme, int32_t V, int32_t F, const int32_t *off_h,
                               const int32_t *fv_h, int32_t K, const int32_t *cv_h,
                               const float *cs_h, void *stream, alsub_mesh_t *out) {
    return alsub_mesh_create_ex(scheme, V, F, off_h, fv_h, K, cv_h, cs_h, nullptr, stream, out);
}

alsub_status alsub_mesh_create_ex(alsub_scheme scheme, int32_t V, int32_t F, const int32_t *off_h,
                                  const int32_t *fv_h, int32_t K, const int32_t *cv_h, const float *cs_h,
                                  const alsub_allocator *allocator, void *stream, alsub_mesh_t *out) {
    return alsub::create_mesh(scheme, V, F, off_h, fv_h, K, cv_h, cs_h, allocator, nullptr, stream, out);
}

alsub_status alsub_mesh_info(alsub_mesh_t h, int32_t *scheme, int64_t *V, int64_t *F, int64_t *nnz,
                             int64_t *K) {
    if (!h) return fail(ALSUB_ERR_INVALID_ARG, "NULL mesh");
    if (scheme) *scheme = h->m.scheme;
    if (V) *V = h->m.V;
    if (F) *F = h->m.F;
    if (nnz) *nnz = h->m.nnz;
    if (K) *K = h->m.K;
    return ALSUB_OK;
}

alsub_status alsub_topology_extract(alsub_topology_t topo, int32_t level, const uint8_t *select_dev,
                                    int32_t rings, void *stream, alsub_mesh_t *out) {
    if (!topo || !out || rings < 1) return fail(ALSUB_ERR_INVALID_ARG, "bad extraction arguments");
    *out = nullptr;
    TopoImpl &T = topo->t;
    if (level < 0 || level > T.levels) return fail(ALSUB_ERR_INVALID_ARG, "bad level");
    if (!T.built) return fail(ALSUB_ERR_INVALID_ARG, "topology not built");
    if (T.scheme == ALSUB_SQRT3)
        return fail(ALSUB_ERR_UNSUPPORTED, "extraction gives an open mesh: sqrt(3) has no boundary rule");
    alsub_mesh_s *h = new (std::nothrow) alsub_mesh_s();
    if (!h) return fail(ALSUB_ERR_OOM, "host allocation failed");
    cudaStream_t s = (cudaStream_t)stream;
    alsub_status st = extract_level(T, level, select_dev, rings, s, h->m);
    long long B = 0;
    bool crease_at_boundary = false;
    if (st == ALSUB_OK) st = mesh_boundary_scan(h->m, s, &B, &crease_at_boundary);
    if (st == ALSUB_OK && crease_at_boundary)
        st = fail(ALSUB_ERR_UNSUPPORTED, "an extracted crease touches the cut");
    if (st != ALSUB_OK) {
        alsub_mesh_destroy(h);
        return st;
    }
    h->m.B = (int)B;
    h->m.src_topo = &T;
    h->m.src_level = level;
    *out = h;
    return ALSUB_OK;
}

alsub_status alsub_mesh_reorder(alsub_mesh_t mesh, void *stream, alsub_mesh_t *out, int32_t *levels) {
    if (!mesh || !out) return fail(ALSUB_ERR_INVALID_ARG, "bad reorder arguments");
    *out = nullptr;
    alsub_mesh_s *h = new (std::nothrow) alsub_mesh_s();
    if (!h) return fail(ALSUB_ERR_OOM, "host allocation failed");
    int lv = 0;
    alsub_status st = reorder_mesh(mesh->m, (cudaStream_t)stream, h->m, &lv);
    if (st != ALSUB_OK) {
        alsub_mesh_destroy(h);
        return st;
    }
    if (levels) *levels = lv;
    *out = h;
    return ALSUB_OK;
}

alsub_status alsub_mesh_arrays(alsub_mesh_t h, const int32_t **off_dev, const int32_t **fv_dev,
                               const int32_t **crease_verts_dev, const float **crease_sharp_dev) {
    if (!h) return fail(ALSUB_ERR_INVALID_ARG, "NULL mesh");
    if (off_dev) *off_dev = h->m.d_off;
    if (fv_dev) *fv_dev = h->m.d_fv;
    if (crease_verts_dev) *crease_verts_dev = h->m.d_cv;
    if (crease_sharp_dev) *crease_sharp_dev = h->m.d_cs;
    return ALSUB_OK;
}

alsub_status alsub_mesh_extract_maps(alsub_mesh_t h, const int32_t **vmap_dev, const int32_t **fmap_dev) {
    if (!h) return fail(ALSUB_ERR_INVALID_ARG, "NULL mesh");
    if (!h->m.d_vmap) return fail(ALSUB_ERR_INVALID_ARG, "mesh has no source maps (not extracted or reordered)");
    if (vmap_dev) *vmap_dev = h->m.d_vmap;
    if (fmap_dev) *fmap_dev = h->m.d_fmap;
    return ALSUB_OK;
}

alsub_status alsub_mesh_gather(alsub_mesh_t h, const float *P_dev, float *out_dev, void *stream) {
    if (!h || !P_dev || !out_dev) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    if (!h->m.d_vmap) return fail(ALSUB_ERR_INVALID_ARG, "mesh has no source maps (not extracted or reordered)");
    gather_rows(h->m.V, h->m.d_vmap, P_dev, out_dev, (cudaStream_t)stream);
    return finish("alsub_mesh_gather");
}

alsub_status alsub_mesh_boundary_edges(alsub_mesh_t h, int64_t *boundary_edges) {
    if (!h || !boundary_edges) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    *boundary_edges = h->m.B;
    return ALSUB_OK;
}

alsub_status alsub_mesh_destroy(alsub_mesh_t h) {
    if (!h) return ALSUB_OK;
    MeshImpl &M = h->m;
    if (M.d_block) {
        dev_free(M.alloc, M.d_block, M.stream);
        M.d_off = M.d_fv = M.d_cv = nullptr;
        M.d_cs = nullptr;
    }
    for (void *p : {(void *)M.d_off, (void *)M.d_fv, (void *)M.d_cv, (void *)M.d_cs, (void *)M.d_vmap,
                    (void *)M.d_fmap})
        if (p) dev_free(M.alloc, p, M.stream);
    delete h;
    return finish("alsub_mesh_destroy");
}

alsub_status alsub_topology_create(alsub_mesh_t mesh, int32_t levels, void *stream,
                                   alsub_topology_t *out) {
    if (!mesh || !out || levels < 0) return fail(ALSUB_ERR_INVALID_ARG, "bad topology arguments");
    *out = nullptr;
    alsub_topology_s *h = new (std::nothrow) alsub_topology_s();
    if (!h) return fail(ALSUB_ERR_OOM, "host allocation failed");
    cudaStream_t s = (cudaStream_t)stream;
    alsub_status st = topo_alloc(h->t, mesh->m, levels, s);
    if (st != ALSUB_OK) {
        h->t.stream = s;
        free_topo(h->t);
        delete h;
        return st;
    }
    st = finish("topology allocation");
    if (st != ALSUB_OK) { free_topo(h->t); delete h; return st; }
    *out = h;
    return ALSUB_OK;
}

alsub_status alsub_refine_topology(alsub_mesh_t mesh, int32_t levels, void *stream,
                                   alsub_topology_t *out) {
    alsub_status st = alsub_topology_create(mesh, levels, stream, out);
    if (st != ALSUB_OK) return st;
    TopoImpl &T = (*out)->t;
    cudaStream_t s = (cudaStream_t)stream;
    level0_build(T, s);
    if (T.s3f) s3f_level0(T, s);
    level0_validate(T, s);
    level0_creases(T, s);
    for (int l = 0; l < levels; l++) {
        step(T, l, true, T.L[l + 1].helpers, nullptr, nullptr, s);
        crease_analyse(T, l, true, s);
    }
    T.built = true;
    return finish("alsub_refine_topology");
}

alsub_status alsub_topology_status(alsub_topology_t h) {
    if (!h) return fail(ALSUB_ERR_INVALID_ARG, "NULL topology");
    TopoImpl &T = h->t;
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, T.status, sizeof(int), cudaMemcpyDeviceToHost, T.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(T.stream);
    if (e != cudaSuccess) return cuda_fail(e, "alsub_topology_status");
    if (st) return fail((alsub_status)st, "device reported %s", alsub_status_string((alsub_status)st));
    return ALSUB_OK;
}

alsub_status alsub_topology_level(alsub_topology_t h, int32_t level, int64_t *V, int64_t *F,
                                  int64_t *nnz, int64_t *E, const int32_t **off, const int32_t **fv) {
    if (!h || level < 0 || level > h->t.levels) return fail(ALSUB_ERR_INVALID_ARG, "bad level");
    const LevelBuf &B = h->t.L[level];
    if (V) *V = B.V;
    if (F) *F = B.F;
    if (nnz) *nnz = B.nnz;
    if (E) *E = B.E;
    if (off) *off = level == 0 ? h->t.mesh->d_off : nullptr;
    if (fv) *fv = B.fv;
    return ALSUB_OK;
}

alsub_status alsub_topology_creases(alsub_topology_t h, int32_t level, int32_t *K,
                                    const int32_t **cv, const float **cs) {
    if (!h || level < 0 || level > h->t.levels || !K) return fail(ALSUB_ERR_INVALID_ARG, "bad level");
    TopoImpl &T = h->t;
    const CreaseList &C = T.L[level].cr;
    int k = 0;
    if (C.cap > 0) {
        T.launches += crease_export(T, level, T.stream);
        cudaError_t e = cudaMemcpyAsync(&k, C.xcount, sizeof(int), cudaMemcpyDeviceToHost, T.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(T.stream);
        if (e != cudaSuccess) return cuda_fail(e, "alsub_topology_creases");
    }
    *K = k;
    if (cv) *cv = C.xverts;
    if (cs) *cs = C.xsig;
    return ALSUB_OK;
}

alsub_status alsub_topology_set_timing(alsub_topology_t h, int32_t capacity) {
    if (!h || capacity < 0) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    TopoImpl &T = h->t;
    CK(cudaStreamSynchronize(T.stream));
    free_events(T);
    if (capacity == 0) return ALSUB_OK;
    size_t n = ((size_t)capacity + 1) * (T.levels + 2);
    T.tev.resize(n);
    for (size_t i = 0; i < n; i++) {
        cudaError_t e = cudaEventCreate(&T.tev[i]);
        if (e != cudaSuccess) {
            T.tev.resize(i);
            free_events(T);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    T.tcap = capacity;
    T.tcalls = 0;
    return ALSUB_OK;
}

alsub_status alsub_topology_timings(alsub_topology_t h, double *ms, int32_t *calls, int64_t *launches) {
    if (!h) return fail(ALSUB_ERR_INVALID_ARG, "NULL topology");
    TopoImpl &T = h->t;
    if (launches) *launches = T.launches;
    T.launches = 0;
    int n = std::min(T.tcalls, T.tcap);
    bool overflow = T.tcalls > T.tcap;
    if (ms) for (int k = 0; k <= T.levels; k++) ms[k] = 0.0;
    for (int c = 0; c < n; c++) {
        size_t b = (size_t)c * (T.levels + 2);
        for (int k = 0; k <= T.levels; k++) {
            CK(cudaEventSynchronize(T.tev[b + k + 1]));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, T.tev[b + k], T.tev[b + k + 1]));
            if (ms) ms[k] += t;
        }
    }
    if (calls) *calls = n;
    T.tcalls = 0;
    if (overflow) return fail(ALSUB_ERR_INVALID_ARG, "more timed calls than the timing capacity");
    return ALSUB_OK;
}

alsub_status alsub_topology_set_edits(alsub_topology_t h, int32_t level, int32_t n, const int32_t *vid_dev,
                                      const float *off_dev, void *stream) {
    if (!h || n < 0 || (n > 0 && (!vid_dev || !off_dev))) return fail(ALSUB_ERR_INVALID_ARG, "bad edit arguments");
    TopoImpl &T = h->t;
    if (level < 1 || level > T.levels) return fail(ALSUB_ERR_INVALID_ARG, "edits apply to levels 1 .. levels");
    cudaStream_t s = (cudaStream_t)stream;
    if (T.edits.size() != (size_t)T.levels + 1) T.edits.assign(T.levels + 1, TopoImpl::LevelEdits());
    TopoImpl::LevelEdits &e = T.edits[level];
    CK(cudaStreamSynchronize(T.stream));          // calls in flight may still read the old edits
    CK(cudaStreamSynchronize(s));
    if (e.vid) dev_free(T.alloc, e.vid, s);
    if (e.off) dev_free(T.alloc, e.off, s);
    e = TopoImpl::LevelEdits();
    drop_graphs(T);                               // captured calls hold the old edit launches
    if (n == 0) return finish("alsub_topology_set_edits");
    CK(dev_malloc(T.alloc, &e.vid, sizeof(int) * (size_t)n, s));
    CK(dev_malloc(T.alloc, &e.off, sizeof(float) * 3 * (size_t)n, s));
    CK(cudaMemcpyAsync(e.vid, vid_dev, sizeof(int) * (size_t)n, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(e.off, off_dev, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, s));
    e.n = n;
    return finish("alsub_topology_set_edits");
}

alsub_status alsub_topology_destroy(alsub_topology_t h) {
    if (!h) return ALSUB_OK;
    for (TopoImpl::LevelEdits &e : h->t.edits) {
        if (e.vid) dev_free(h->t.alloc, e.vid, h->t.stream);
        if (e.off) dev_free(h->t.alloc, e.off, h->t.stream);
    }
    free_hostio(h->t);
    free_events(h->t);
    drop_graphs(h->t);
    if (h->t.cap) cudaStreamDestroy(h->t.cap);
    free_side(h->t);
    free_topo(h->t);
    delete h;
    return finish("alsub_topology_destroy");
}

alsub_status alsub_refine_vertices_scratch_bytes(alsub_topology_t h, size_t *bytes) {
    if (!h || !bytes) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    *bytes = h->t.scratch_bytes;
    return ALSUB_OK;
}

alsub_status alsub_plan_bytes(alsub_scheme scheme, int32_t V, int32_t F, int32_t nnz, int32_t B, int32_t K,
                              float sigma_max, int32_t levels, size_t *bytes) {
    if (!bytes || K < 0 || !(sigma_max >= 0.f)) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    std::vector<int64_t> c(4 * ((size_t)std::max(levels, 0) + 1));
    alsub_status st = alsub_plan_open(scheme, V, F, nnz, B, levels, c.data());
    if (st != ALSUB_OK) return st;
    MeshImpl M;
    M.scheme = scheme; M.V = V; M.F = F; M.nnz = nnz; M.B = B;
    // sqrt(3) keeps infinitely sharp creases only: num_creases counts those
    M.K = scheme == ALSUB_SQRT3 ? (isinf(sigma_max) ? K : 0) : K;
    M.sigma_max = M.K ? sigma_max : 0.f;
    TopoImpl T;
    T.dry = true;
    st = topo_alloc(T, M, levels, nullptr);
    if (st != ALSUB_OK) return st;
    *bytes = T.bytes;
    return ALSUB_OK;
}

alsub_status alsub_topology_bytes(alsub_topology_t h, size_t *bytes) {
    if (!h || !bytes) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    *bytes = h->t.bytes;
    return ALSUB_OK;
}

alsub_status alsub_refine_vertices(alsub_topology_t h, const float *P0, float *PL, void *scratch,
                                   void *stream) {
    if (!h || !P0 || !PL) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    return refine_call(h->t, P0, PL, scratch, (cudaStream_t)stream);
}

alsub_status alsub_subdivide_host(alsub_topology_t h, const float *P0_host, float *PL_host, void *stream) {
    if (!h || !P0_host || !PL_host) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    TopoImpl &T = h->t;
    alsub_status st = ensure_hostio(T);
    if (st != ALSUB_OK) return st;
    TopoImpl::HostIO &io = T.io;
    const int b = (int)(io.calls & 1);
    const size_t n0 = 12 * (size_t)T.L[0].V, nl = 12 * (size_t)T.L[T.levels].V;
    // the staging buffer was last read by the upload of call k - 2
    CK(cudaEventSynchronize(io.up[b]));
    memcpy(io.hP0[b], P0_host, n0);
    CK(cudaMemcpyAsync(io.dP0, io.hP0[b], n0, cudaMemcpyHostToDevice, io.cs));
    CK(cudaEventRecord(io.up[b], io.cs));
    CK(cudaStreamWaitEvent(io.cs, io.copied[b], 0));     // output buffer b: call k - 2's download done
    st = run_call(T, 1, io.dP0, io.dPL[b], nullptr, io.cs, subdivide_body, true);   // the handle's buffers recur
    if (T.tcap) T.tcalls++;
    if (st != ALSUB_OK) return st;
    T.built = true;
    CK(cudaEventRecord(io.done[b], io.cs));
    CK(cudaStreamWaitEvent(io.ds, io.done[b], 0));
    CK(cudaMemcpyAsync(PL_host, io.dPL[b], nl, cudaMemcpyDeviceToHost, io.ds));
    CK(cudaEventRecord(io.copied[b], io.ds));
    CK(cudaStreamWaitEvent((cudaStream_t)stream, io.copied[b], 0));
    io.calls++;
    return ALSUB_OK;
}

alsub_status alsub_subdivide(alsub_topology_t h, const float *P0, float *PL, void *scratch,
                             void *stream) {
    if (!h || !P0 || !PL) return fail(ALSUB_ERR_INVALID_ARG, "bad arguments");
    TopoImpl &T = h->t;
    alsub_status st = run_call(T, 1, P0, PL, scratch, (cudaStream_t)stream, subdivide_body);
    if (T.tcap) T.tcalls++;
    if (st == ALSUB_OK) T.built = true;
    return st;
}

}  // extern "C"
