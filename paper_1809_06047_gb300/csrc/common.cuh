// Device-side helpers shared by the libalsub kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "alsub.h"
#include "internal.h"

namespace alsub {

// Largest vertex valence a ring walk follows before it reports ALSUB_ERR_UNSUPPORTED.
constexpr int kMaxValence = 1024;
// Largest number of refinement levels of one topology (int32 counts end far earlier in practice).
constexpr int kMaxLevels = 16;
constexpr int kBlock = 256;

// Latch the first device-side error of a handle; later kernels test it and return early.
__device__ __forceinline__ void set_status(int *st, int code) {
    if (st) atomicCAS(st, 0, code);
}
__device__ __forceinline__ bool failed(const int *st) { return st && *(volatile const int *)st != 0; }

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 &operator+=(float3 &a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }

// Positions are packed float[3 * V].
__device__ __forceinline__ float3 ldp(const float *__restrict__ P, int v) {
    const float *p = P + 3 * (size_t)v;
    return f3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
}
// Plain (coherent) load: used where the same kernel, or an earlier one in the same stream,
// wrote the value.
__device__ __forceinline__ float3 ldp_rw(const float *P, int v) {
    const float *p = P + 3 * (size_t)v;
    return f3(p[0], p[1], p[2]);
}
__device__ __forceinline__ void stp(float *P, int v, float3 a) {
    float *p = P + 3 * (size_t)v;
    p[0] = a.x; p[1] = a.y; p[2] = a.z;
}

// Positions of intermediate levels are padded to 16-byte rows (float4, w unused) so a vertex is one
// vector load or store; the caller's input and output levels stay packed xyz. `s4` selects the
// layout of a buffer.
__device__ __forceinline__ float3 ldpv(const float *__restrict__ P, int v, bool s4) {
    if (s4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(P) + v);
        return f3(q.x, q.y, q.z);
    }
    return ldp(P, v);
}
__device__ __forceinline__ float3 ldpv_rw(const float *P, int v, bool s4) {
    if (s4) {
        const float4 q = reinterpret_cast<const float4 *>(P)[v];
        return f3(q.x, q.y, q.z);
    }
    return ldp_rw(P, v);
}
__device__ __forceinline__ void stpv(float *P, int v, float3 a, bool s4) {
    if (s4) reinterpret_cast<float4 *>(P)[v] = make_float4(a.x, a.y, a.z, 0.f);
    else stp(P, v, a);
}

// Corner arithmetic of quads (levels >= 1 of Catmull-Clark) and triangles (Loop, sqrt(3)).
__device__ __forceinline__ int quad_next(int x) { return (x & ~3) | ((x + 1) & 3); }
__device__ __forceinline__ int quad_prev(int x) { return (x & ~3) | ((x + 3) & 3); }
__device__ __forceinline__ int tri_next(int x) { int j = x % 3; return x - j + (j == 2 ? 0 : j + 1); }
__device__ __forceinline__ int tri_prev(int x) { int j = x % 3; return x - j + (j == 0 ? 2 : j - 1); }

// Level-0 (general polygon) adjacency, built on the device from the input face table.
struct Level0 {
    const int *off;   // F0 + 1 face offsets
    const int *fv;    // nnz0 vertex of each corner
    const int *cf;    // corner -> face
    const int *nx;    // next corner in the face
    const int *pv;    // previous corner in the face
    const int *tw;    // twin corner (the corner of the same edge in the other face)
    const int *ce;    // edge id of each corner
    const int *own;   // 1 if the corner owns its edge (start vertex < end vertex)
    const int *vc;    // designated (smallest) outgoing corner of each vertex
    const int *rn;    // ring step twin(prev(x)): the next outgoing corner around the start vertex
    const int *rec = nullptr;   // Catmull-Clark ring records of level 0 (kRec* below), or null
};

// Ring record of level-0 corner c (16 ints at rec + 16 c) for the vertices that refined levels
// >= 2 cannot classify by index arithmetic alone (those born on levels 0 and 1):
//   [kRecVertex]  the vertex fv[c] when c is its designated corner: its valence n (1 .. 8, the
//                 ring's corners in walk order x <- twin(prev(x)) at [8, 8 + n)), kRecOpen on the
//                 boundary, kRecLong for a longer ring (walked instead); 0 elsewhere
//   [kRecEdge]    the edge point of c's edge when c owns it: the twin t of c (kRecOpen for a
//                 boundary edge), with [2] = next(t) and [3] = next(c); -1 when c does not own it
//   [4]           the face point of c's face when c is its first corner: the face's order; else 0
constexpr int kRecInts = 16;
constexpr int kRecVertex = 0, kRecEdge = 1, kRecFace = 4, kRecRing = 8, kRecMaxRing = 8;
constexpr int kRecOpen = -2, kRecLong = -3;

// Corner accessors used by the ring walks of the crease kernels. Each gives next / prev corner
// in the face, the ring step twin(prev), twin, edge id and start vertex of a corner.
struct AccL0 {
    static constexpr int kRound = 8;
    Level0 z;
    __device__ int next(int x) const { return __ldg(z.nx + x); }
    __device__ int prev(int x) const { return __ldg(z.pv + x); }
    __device__ int ring(int x) const { return __ldg(z.rn + x); }
    __device__ int twin(int x) const { return __ldg(z.tw + x); }
    __device__ int edge(int x) const { return __ldg(z.ce + x); }
    __device__ int vtx(int x) const { return __ldg(z.fv + x); }
};
struct AccQuad {
    static constexpr int kRound = 4;
    const int *fv, *tw, *ce;
    __device__ int next(int x) const { return quad_next(x); }
    __device__ int prev(int x) const { return quad_prev(x); }
    __device__ int ring(int x) const { return __ldg(tw + quad_prev(x)); }
    __device__ int twin(int x) const { return __ldg(tw + x); }
    __device__ int edge(int x) const { return __ldg(ce + x); }
    __device__ int vtx(int x) const { return __ldg(fv + x); }
};

__device__ __forceinline__ int4 ld4(const int *p) { return __ldg(reinterpret_cast<const int4 *>(p)); }
__device__ __forceinline__ void st4(int *p, int4 v) { *reinterpret_cast<int4 *>(p) = v; }
__device__ __forceinline__ int comp(int4 v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// ---- designated corners. Every vertex of a level is gathered (or gets its operator row) from
// exactly one of its corners. Each test follows the vertex back to the level where it was
// created: an old vertex inherits from its parent corner, an edge point is designated at a child
// of its edge's owner corner, a face point at a child of its face's first corner; level-0 vertices
// use their smallest outgoing corner (vc).

// Catmull-Clark, corner x of level l (levels >= 1 are quads: child k of parent corner c is 4c+k).
__device__ __forceinline__ bool cc_vown(int l, int x, const Level0 &z) {
    while (l > 0) {
        int k = x & 3, c = x >> 2;
        if (k == 0) { x = c; --l; continue; }
        if (k == 3) return false;
        if (k == 1) return l > 1 ? ((c & 3) < 2) : (__ldg(z.own + c) != 0);
        return l > 1 ? ((c & 3) == 0) : (c == __ldg(z.off + __ldg(z.cf + c)));
    }
    return __ldg(z.vc + __ldg(z.fv + x)) == x;
}

// Loop: does corner x of level l own its edge?
__device__ __forceinline__ bool loop_own(int l, int x, const Level0 &z) {
    if (l == 0) return __ldg(z.own + x) != 0;
    int g = x / 3, i = x - 3 * g;
    return (g & 3) < 3 && i < 2;
}

// The same two tests with the corner given as (triangle g, corner i): no division by 3. A corner-0
// vertex of a corner child is corner j of the parent triangle g >> 2, i.e. (g >> 2, j) again.
__device__ __forceinline__ bool loop_own_gi(int l, int g, int i, const Level0 &z) {
    if (l == 0) return __ldg(z.own + 3 * g + i) != 0;
    return (g & 3) < 3 && i < 2;
}
__device__ __forceinline__ bool loop_vown_gi(int l, int g, int i, const Level0 &z) {
    while (l > 0) {
        const int r = g >> 2, j = g & 3;
        if (j == 3 || i == 2) return false;
        if (i == 0) { g = r; i = j; --l; continue; }
        return loop_own_gi(l - 1, r, j, z);
    }
    return __ldg(z.vc + __ldg(z.fv + 3 * g + i)) == 3 * g + i;
}

// Loop: corner i of child j of triangle r is 3(4r + j) + i.
__device__ __forceinline__ bool loop_vown(int l, int x, const Level0 &z) {
    while (l > 0) {
        int g = x / 3, i = x - 3 * g, r = g >> 2, j = g & 3;
        if (j == 3 || i == 2) return false;
        if (i == 0) { x = 3 * r + j; --l; continue; }
        return loop_own(l - 1, 3 * r + j, z);
    }
    return __ldg(z.vc + __ldg(z.fv + x)) == x;
}

// Per-corner edge ids and twins of a Loop or sqrt(3) level: read from the level's arrays, or, for a
// level that does not store them, derived from its parent level's arrays by the same child rules
// the build writes them with (one load per derived value; some need none).
//   Loop, corner i of child j of parent triangle R (corner x = 3(4R + j) + i):
//     j < 3, i = 0: edge 2 e_R(j) + (R's corner j owns its edge ? 0 : 1),
//                   twin 3(4s + (k == 2 ? 0 : k + 1)) + 2 with tw_R(j) = 3s + k;
//     j < 3, i = 1: edge 2E + 3R + j, twin 3(4R + 3) + (j + 2) % 3;
//     j < 3, i = 2: edge 2 e_R(j - 1) + (owns ? 1 : 0), twin 3 tw_R(j - 1) rounded to its
//                   child 0 (3(4s + k));
//     j = 3:        edge 2E + 3R + (i + 1) % 3, twin 3(4R + (i + 1) % 3) + 1;
//   sqrt(3), corner k of child c (the child of parent corner c, x = 3c + k):
//     k = 0: 3 next(tw(c)) + 2;  k = 1: 3 tw(c) + 1;  k = 2: 3 tw(prev c).
struct TriLevel {
    const int *ce = nullptr, *tw = nullptr;    // this level's arrays (stored)
    const int *pce = nullptr, *ptw = nullptr;  // the parent level's arrays (derived)
    int E2p = 0;                               // 2 E of the parent level
    int lp = 0;                                // parent level
    bool derive = false, sqrt3 = false;
    Level0 z;

    // Branch-free: the lanes of a warp take different cases, so each case must not issue a load
    // of its own (one predicated load, then selects).
    __device__ int twin(int x) const {
        if (!derive) return __ldg(tw + x);
        if (sqrt3) {
            const int c = x / 3, k = x - 3 * c;
            const int t = __ldg(ptw + (k == 2 ? tri_prev(c) : c));
            return k == 0 ? 3 * tri_next(t) + 2 : (k == 1 ? 3 * t + 1 : 3 * t);
        }
        const int g = x / 3, i = x - 3 * g, R = g >> 2, j = g & 3;
        const int jm = j == 0 ? 2 : j - 1;
        const bool need = j != 3 && i != 1;
        const int t = need ? __ldg(ptw + 3 * R + (i == 0 ? j : jm)) : 0;
        const int s = t / 3, k = t - 3 * s;
        const int fromParent = t < 0 ? -1 : (i == 0 ? 3 * (4 * s + (k == 2 ? 0 : k + 1)) + 2 : 3 * (4 * s + k));
        const int interior = j == 3 ? 3 * (4 * R + (i == 2 ? 0 : i + 1)) + 1 : 3 * (4 * R + 3) + jm;
        return need ? fromParent : interior;          // -1: the half of a boundary edge
    }
    // Loop only (sqrt(3) has no edge ids); edge_gi takes corner i of triangle g
    __device__ int edge(int x) const;
    __device__ int edge_gi(int g, int i) const;
};

// sqrt(3): corner k of child c (the child of parent corner c) is 3c + k.
__device__ __forceinline__ bool sqrt3_vown(int l, int x, const Level0 &z) {
    while (l > 0) {
        int c = x / 3, k = x - 3 * c;
        if (k == 0) { x = c; --l; continue; }
        if (k == 1) return false;
        return c % 3 == 0;
    }
    return __ldg(z.vc + __ldg(z.fv + x)) == x;
}

__device__ __forceinline__ int TriLevel::edge(int x) const {
    if (!derive) return __ldg(ce + x);
    const int g = x / 3;
    return edge_gi(g, x - 3 * g);
}
__device__ __forceinline__ int TriLevel::edge_gi(int g, int i) const {
    if (!derive) return __ldg(ce + 3 * g + i);
    const int R = g >> 2, j = g & 3;
    const bool need = j != 3 && i != 1;
    const int pc = 3 * R + (i == 0 ? j : (j == 0 ? 2 : j - 1));
    const int pe = need ? __ldg(pce + pc) : 0;
    const bool own = need && loop_own_gi(lp, R, i == 0 ? j : (j == 0 ? 2 : j - 1), z);
    const int fromParent = 2 * pe + (i == 0 ? (own ? 0 : 1) : (own ? 1 : 0));
    const int interior = E2p + 3 * R + (j == 3 ? (i == 2 ? 0 : i + 1) : j);
    return need ? fromParent : interior;
}

struct AccTri {
    static constexpr int kRound = 8;
    const int *fv;
    TriLevel t;
    __device__ int next(int x) const { return tri_next(x); }
    __device__ int prev(int x) const { return tri_prev(x); }
    __device__ int ring(int x) const { return t.twin(tri_prev(x)); }
    __device__ int twin(int x) const { return t.twin(x); }
    __device__ int edge(int x) const { return t.edge(x); }
    __device__ int vtx(int x) const { return __ldg(fv + x); }
};

// Crease hash table (CreaseList::tab): linear probing from a multiplicative hash.
// The table holds 2^k int2 slots (key = edge id, -1 = empty; value = sharpness bits) at load
// factor <= 1/4, probed linearly in aligned pairs: bucket b is slots 2b, 2b + 1, read by one
// 16-byte load, then bucket b + 1 and so on. Inserts fill the same sequence, so an empty slot ends
// a search.
__device__ __forceinline__ unsigned crease_bucket(int e, int shift) {
    return shift >= 31 ? 0u : ((unsigned)e * 2654435761u) >> (shift + 1);
}
__device__ __forceinline__ float crease_lookup(const CreaseList &C, int e) {
    const int4 *__restrict__ t = reinterpret_cast<const int4 *>(C.tab);
    const unsigned bmask = (unsigned)C.hmask >> 1;
    unsigned b = crease_bucket(e, C.hshift);
    for (unsigned probe = 0; probe <= bmask; probe++) {
        const int4 q = __ldg(t + b);
        if (q.x == e) return __int_as_float(q.y);
        if (q.x < 0) return 0.f;
        if (q.z == e) return __int_as_float(q.w);
        if (q.z < 0) return 0.f;
        b = (b + 1) & bmask;
    }
    return 0.f;
}
// A lookup whose first bucket b was loaded already (q): resolved from it, probing on only when the
// bucket holds two other edges. Lets a thread issue the first probes of many lookups at once.
__device__ __forceinline__ float crease_resolve(const CreaseList &C, int e, unsigned b, int4 q) {
    if (q.x == e) return __int_as_float(q.y);
    if (q.x < 0) return 0.f;
    if (q.z == e) return __int_as_float(q.w);
    if (q.z < 0) return 0.f;
    const int4 *__restrict__ t = reinterpret_cast<const int4 *>(C.tab);
    const unsigned bmask = (unsigned)C.hmask >> 1;
    b = (b + 1) & bmask;
    for (unsigned probe = 0; probe < bmask; probe++) {
        const int4 r = __ldg(t + b);
        if (r.x == e) return __int_as_float(r.y);
        if (r.x < 0) return 0.f;
        if (r.z == e) return __int_as_float(r.w);
        if (r.z < 0) return 0.f;
        b = (b + 1) & bmask;
    }
    return 0.f;
}
// Returns false when the edge was already in the table.
__device__ __forceinline__ bool crease_insert(const CreaseList &C, int e, float s) {
    const unsigned bmask = (unsigned)C.hmask >> 1;
    unsigned b = crease_bucket(e, C.hshift);
    for (unsigned probe = 0; probe <= bmask; probe++) {
        for (int h = 0; h < 2; h++) {
            int2 *slot = C.tab + 2 * b + h;
            const int old = atomicCAS(&slot->x, -1, e);
            if (old == -1) {
                slot->y = __float_as_int(s);
                return true;
            }
            if (old == e) return false;
        }
        b = (b + 1) & bmask;
    }
    return false;
}

inline unsigned grid_for(long long n, int block = kBlock) {
    long long g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

// Programmatic dependent launch. A kernel launched by launch_pdl may be scheduled while the kernel
// before it in the stream is still draining (its blocks take the SMs that free up), so its start
// is not a launch gap behind the previous kernel's last block. Such a kernel calls pdl_wait()
// before its first memory access: it returns once the previous grid has completed and its
// writes are visible (and at once when there is no such dependency). pdl_trigger() lets the next
// kernel launch as soon as every block of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace alsub
