// Creases (Sec. 3.3) for Catmull-Clark and Loop.
//
// The crease matrix C_l is kept as a list of tagged edges, plus an open-addressing hash table
// (edge id -> sharpness) for the O(1) lookups of the ring walks. For
// each crease end vertex one ring walk computes the crease valency k (Eq. CC_crease_valency) and
// the sharpness sum in the same pass (the fused k / s SpMV of Sec. 4.4), so s = S / k
// (Eq. CC_crease_vsharpness).
//
// Per level, an analysis kernel walks the rings (it needs only the level's adjacency, so it can run
// beside the level's eval) and keeps each entry's result; a fix kernel then applies the rules:
//  fix (after the smooth eval of the level, Fig. module_creases) overwrites
//    the edge point of a crease: sigma >= 1 -> midpoint, else (1 - sigma) smooth + sigma midpoint;
//    a crease vertex with k >= 2: w sharp + (1 - w) smooth, w = min(s, 1), sharp =
//    (p_a + 6 p + p_b) / 8 for k == 2 and p for k >= 3. Exactly one crease thread writes a vertex:
//    the one whose outgoing corner at that vertex is the smallest among the vertex's creases;
//  inherit (Sec. 3.3) gives each crease's two halves the sharpness max((sigma_o + 3 sigma) / 4 - 1,
//    0) (the Chaikin-style rule), evaluated with correctly rounded FP32 operations in a fixed
//    order. The halves go straight to entries 2i, 2i + 1 of the next level's list (so its order
//    follows the input order of level 0) and the live ones into its hash table; halves that
//    decayed to 0 stay as inert entries. The paper's count-then-fill compaction is done only when
//    a level's list is exported (crease_export).
#include <float.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

struct CreaseArgs {
    int epbase;                 // id of edge point 0 in level l + 1 (CC: V + F, Loop: V)
    int child_tri;              // 1: Loop child-corner mapping, 0: Catmull-Clark
    CreaseList in;
    CreaseList out;             // the next level's list
    int *flags;
    const float *P;
    float *Pn;
    bool in4, out4;             // level l / l + 1 positions in padded float4 rows
    int *status;
};

struct EndInfo {
    int k;          // incident creases
    float S;        // their sharpness sum, in ring order from the start corner
    int n1, n2;     // the first two crease neighbours
    float s1, s2;
    int minc;       // smallest outgoing crease corner at the vertex
};

__device__ __forceinline__ void end_init(EndInfo &r) {
    r.k = 0; r.S = 0.f; r.n1 = r.n2 = -1; r.s1 = r.s2 = 0.f; r.minc = 0x7fffffff;
}
__device__ __forceinline__ void end_add(EndInfo &r, int y, float sy, int nb) {
    if (!(sy > 0.f)) return;
    if (r.k == 0) { r.n1 = nb; r.s1 = sy; }
    else if (r.k == 1) { r.n2 = nb; r.s2 = sy; }
    r.k++;
    r.S += sy;
    r.minc = min(r.minc, y);
}

// Both end vertices of a crease in one pass. The rings are walked in lockstep, kW corners per
// round (4 for quads, 8 for the level-0 polygons and triangles): first the twin chain of the round (the only dependent loads), then the edge-id, table
// and neighbour loads of all kW corners, which are independent of one another. Crease valency k,
// sharpness sum S (added in ring order from the start corner), the first two crease neighbours
// and the smallest crease corner come out exactly as a one-corner-at-a-time walk gives them.
template <class Acc>
__device__ void analyse2(const Acc &A, const CreaseList &C, int sa, int sb, EndInfo &ra, EndInfo &rb,
                         int *status) {
    constexpr int kW = Acc::kRound;         // valence of a typical vertex: one round
    end_init(ra);
    end_init(rb);
    int ya = sa, yb = sb;
    bool da = false, db = false;
    for (int steps = 0; !(da && db) && steps < kMaxValence; steps += kW) {
        int ca[kW], cb[kW];
        bool ua[kW], ub[kW];
#pragma unroll
        for (int q = 0; q < kW; q++) {
            ua[q] = !da; ca[q] = ya;
            ub[q] = !db; cb[q] = yb;
            if (!da) { ya = A.ring(ya); da = ya == sa; }
            if (!db) { yb = A.ring(yb); db = yb == sb; }
        }
        // the round's lookups: every edge id, then every first bucket, then their resolution (a
        // lookup only probes on past a bucket of two other edges), so they share round trips
        const int4 *__restrict__ tab = reinterpret_cast<const int4 *>(C.tab);
        int ea[kW], eb[kW];
        int na[kW], nb[kW];
#pragma unroll
        for (int q = 0; q < kW; q++) {
            ea[q] = ua[q] ? A.edge(ca[q]) : 0;
            eb[q] = ub[q] ? A.edge(cb[q]) : 0;
            na[q] = ua[q] ? A.vtx(A.next(ca[q])) : -1;
            nb[q] = ub[q] ? A.vtx(A.next(cb[q])) : -1;
        }
        int4 qa[kW], qb[kW];
#pragma unroll
        for (int q = 0; q < kW; q++) {
            qa[q] = ua[q] ? __ldg(tab + crease_bucket(ea[q], C.hshift)) : make_int4(-1, 0, -1, 0);
            qb[q] = ub[q] ? __ldg(tab + crease_bucket(eb[q], C.hshift)) : make_int4(-1, 0, -1, 0);
        }
        float fa[kW], fb[kW];
#pragma unroll
        for (int q = 0; q < kW; q++) {
            fa[q] = ua[q] ? crease_resolve(C, ea[q], crease_bucket(ea[q], C.hshift), qa[q]) : 0.f;
            fb[q] = ub[q] ? crease_resolve(C, eb[q], crease_bucket(eb[q], C.hshift), qb[q]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kW; q++) {
            if (ua[q]) end_add(ra, ca[q], fa[q], na[q]);
            if (ub[q]) end_add(rb, cb[q], fb[q], nb[q]);
        }
    }
    if (!(da && db)) set_status(status, ALSUB_ERR_UNSUPPORTED);
}

__device__ __forceinline__ float chaikin(float so, float s) {
    float t = __fmul_rn(3.0f, s);
    float u = __fadd_rn(so, t);
    float w = __fmul_rn(u, 0.25f);
    float y = __fsub_rn(w, 1.0f);
    return y > 0.f ? y : 0.f;
}

__device__ __forceinline__ int child_corner(int x, int tri) {
    if (!tri) return 4 * x;                 // Catmull-Clark: corner 0 of child quad x
    int r = x / 3, j = x - 3 * r;           // Loop: corner 0 of child j of triangle r
    return 3 * (4 * r + j);
}

// Analysis of one crease entry: both end vertices' crease valency, sharpness sum, first two crease
// neighbours and whether this entry designates the vertex (kept in info for the fix), and with
// INHERIT the entry's two halves in the next level's list and table.
template <class Acc, bool INHERIT>
__global__ void __launch_bounds__(kBlock) k_crease_analyse(Acc A, CreaseArgs a, int cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    // the entry is read together with the count (slots past the count are allocated, unused)
    const int e = a.in.edge[i], o = a.in.own[i];
    const float s = a.in.sig[i];
    const int K = failed(a.status) ? 0 : *a.in.count;
    if (INHERIT && i == 0) *a.out.count = 2 * K;
    if (i >= K) return;
    if (!(s > 0.f)) {
        // an inherited zero: no crease any more; its children stay inert entries
        a.in.info[2 * i] = make_int4(0, 0, -1, -1);
        a.in.info[2 * i + 1] = make_int4(0, 0, -1, -1);
        if (INHERIT) {
            for (int h = 0; h < 2; h++) {
                a.out.edge[2 * i + h] = 2 * e + h;
                a.out.own[2 * i + h] = 0;
                a.out.sig[2 * i + h] = 0.f;
                a.out.verts[4 * i + 2 * h] = 0;
                a.out.verts[4 * i + 2 * h + 1] = 0;
            }
        }
        return;
    }
    const int t = A.twin(o);
    const int va = A.vtx(o);
    // the list holds the entry's two endpoints (in either order): the one that is not v_o's
    const int first = a.in.verts[2 * i], second = a.in.verts[2 * i + 1];
    const int vb = first == va ? second : first;
    EndInfo ra, rb;
    analyse2(A, a.in, o, t, ra, rb, a.status);
    const int4 ia = make_int4(ra.k | (ra.minc == o ? 1 << 16 : 0), __float_as_int(ra.S), ra.n1, ra.n2);
    const int4 ib = make_int4(rb.k | (rb.minc == t ? 1 << 16 : 0), __float_as_int(rb.S), rb.n1, rb.n2);
    const bool swap = first != va;          // the odd half of a parent crease lists (ep, v_t)
    a.in.info[2 * i] = swap ? ib : ia;
    a.in.info[2 * i + 1] = swap ? ia : ib;
    if (INHERIT) {
        const int ep = a.epbase + e;
        float oa = s, ob = s;
        if (ra.k == 2) { float x = ra.n1 == vb ? ra.s2 : ra.s1; if (isfinite(x)) oa = x; }
        if (rb.k == 2) { float x = rb.n1 == va ? rb.s2 : rb.s1; if (isfinite(x)) ob = x; }
        const float ca = chaikin(oa, s), cb = chaikin(ob, s);
        // the half at v_o is 2e (o owns e), the half at v_t is 2e + 1
        a.out.edge[2 * i] = 2 * e;
        a.out.own[2 * i] = child_corner(o, a.child_tri);
        a.out.sig[2 * i] = ca;
        a.out.verts[4 * i] = va;
        a.out.verts[4 * i + 1] = ep;
        a.out.edge[2 * i + 1] = 2 * e + 1;
        a.out.own[2 * i + 1] = child_corner(t, a.child_tri);
        a.out.sig[2 * i + 1] = cb;
        a.out.verts[4 * i + 2] = ep;
        a.out.verts[4 * i + 3] = vb;
        if (ca > 0.f) crease_insert(a.out, 2 * e, ca);
        if (cb > 0.f) crease_insert(a.out, 2 * e + 1, cb);
    }
}

// Fix of one crease entry from its stored analysis: the crease edge point, and each end vertex the
// entry designates (exactly one crease per crease vertex does).
__global__ void __launch_bounds__(kBlock) k_crease_fix(CreaseArgs a, int cap) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    const int e = a.in.edge[i];
    const float s = a.in.sig[i];
    const int va = a.in.verts[2 * i], vb = a.in.verts[2 * i + 1];
    const int4 ia = a.in.info[2 * i], ib = a.in.info[2 * i + 1];
    const int K = failed(a.status) ? 0 : *a.in.count;
    if (i >= K || !(s > 0.f)) return;
    const int ep = a.epbase + e;
    const float3 pa = ldpv(a.P, va, a.in4), pb = ldpv(a.P, vb, a.in4);
    const float3 mid = 0.5f * (pa + pb);
    if (s >= 1.0f) stpv(a.Pn, ep, mid, a.out4);
    else stpv(a.Pn, ep, (1.0f - s) * ldpv_rw(a.Pn, ep, a.out4) + s * mid, a.out4);
    const int4 info[2] = {ia, ib};
    const int verts[2] = {va, vb};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int k = info[h].x & 0xffff;
        if (!(info[h].x >> 16) || k < 2) continue;
        const int v = verts[h];
        const float sv = __int_as_float(info[h].y) / (float)k;
        const float w = sv < 1.0f ? sv : 1.0f;
        const float3 p = h == 0 ? pa : pb;
        const float3 sharp =
            k == 2 ? 0.125f * (ldpv(a.P, info[h].z, a.in4) + 6.0f * p + ldpv(a.P, info[h].w, a.in4)) : p;
        stpv(a.Pn, v, w * sharp + (1.0f - w) * ldpv_rw(a.Pn, v, a.out4), a.out4);
    }
}

__global__ void k_export_flags(int n, const CreaseList c, int *flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = i < *c.count && c.sig[i] > 0.f;
}

__global__ void k_export(int n, const int *__restrict__ flags, const int *__restrict__ pos, CreaseList c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    const int k = pos[i];
    c.xverts[2 * k] = c.verts[2 * i];
    c.xverts[2 * k + 1] = c.verts[2 * i + 1];
    c.xsig[k] = c.sig[i];
}

template <class F>
void with_acc(TopoImpl &T, int l, F f) {
    LevelBuf &A = T.L[l];
    if (l == 0) {
        AccL0 acc;
        acc.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0, T.rn0};
        f(acc);
    } else if (T.scheme == ALSUB_CATMULL_CLARK) {
        f(AccQuad{A.fv, A.tw, A.ce});
    } else {
        f(AccTri{A.fv, tri_level(T, l)});
    }
}

CreaseArgs base_args(TopoImpl &T, int l) {
    LevelBuf &A = T.L[l];
    CreaseArgs a;
    a.epbase = (int)(T.scheme == ALSUB_CATMULL_CLARK ? A.V + A.F : A.V);
    a.child_tri = T.scheme == ALSUB_LOOP;
    a.in = A.cr;
    a.out = T.L[l + 1 <= T.levels ? l + 1 : l].cr;
    a.flags = T.flags;
    a.P = nullptr; a.Pn = nullptr;
    a.status = T.status;
    a.in4 = l > 0;
    a.out4 = l + 1 < T.levels;
    return a;
}

}  // namespace

void crease_table_clear(const CreaseList &C, cudaStream_t s) {
    if (C.tab) cudaMemsetAsync(C.tab, 0xff, sizeof(int2) * ((size_t)C.hmask + 1), s);
}

bool crease_alive(const TopoImpl &T, int l) {
    return T.scheme != ALSUB_SQRT3 && l <= T.levels && T.L[l].cr.cap > 0;
}

void crease_analyse(TopoImpl &T, int l, bool inherit, cudaStream_t s) {
    CreaseList *dst = l + 1 <= T.levels ? &T.L[l + 1].cr : nullptr;
    if (inherit && dst && dst->cap == 0) inherit = false;   // all creases have decayed: level l + 1
                                                              // has none (its count stays 0)
    if (!dst) inherit = false;
    if (!crease_alive(T, l)) return;
    if (inherit) crease_table_clear(*dst, s);
    CreaseArgs a = base_args(T, l);
    if (inherit) a.out = *dst;
    const int cap = (int)T.L[l].cr.cap;
    const unsigned g = grid_for(cap);
    with_acc(T, l, [&](auto acc) {
        using A = decltype(acc);
        if (inherit) k_crease_analyse<A, true><<<g, kBlock, 0, s>>>(acc, a, cap);
        else k_crease_analyse<A, false><<<g, kBlock, 0, s>>>(acc, a, cap);
    });
    T.launches += 1;
}

void crease_fix(TopoImpl &T, int l, const float *P, float *Pn, cudaStream_t s) {
    if (!crease_alive(T, l) || l >= T.levels) return;
    CreaseArgs a = base_args(T, l);
    a.P = P;
    a.Pn = Pn;
    const int cap = (int)T.L[l].cr.cap;
    launch_pdl(k_crease_fix, grid_for(cap), kBlock, s, a, cap);
    T.launches += 1;
}

int crease_export(TopoImpl &T, int l, cudaStream_t s) {
    if (T.s3f) return s3f_export(T, l, s);
    CreaseList &C = T.L[l].cr;
    if (C.cap == 0) return 0;
    const long long n = C.cap;
    k_export_flags<<<grid_for(n), kBlock, 0, s>>>((int)n, C, T.flags);
    int k = 2 + scan_exclusive(T.flags, T.pos, n, C.xcount, nullptr, T.scan_tmp, s);
    k_export<<<grid_for(n), kBlock, 0, s>>>((int)n, T.flags, T.pos, C);
    return k;
}

}  // namespace alsub
