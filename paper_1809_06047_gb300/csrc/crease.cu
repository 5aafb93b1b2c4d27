// Creases (Sec. 3.3) for Catmull-Clark and Loop.
//
// The crease matrix C_l is kept as a list of tagged edges sorted by edge id; a crease is looked up
// by binary search. For each crease end vertex the ring walk computes the crease valency k (Eq.
// CC_crease_valency) and the sharpness sum in the same pass (the fused k / s SpMV of Sec. 4.4),
// so s = S / k (Eq. CC_crease_vsharpness).
//
// crease_fix runs after the smooth eval of a level and overwrites (Fig. module_creases):
//   the edge point of a crease: sigma >= 1 -> midpoint, else (1 - sigma) smooth + sigma midpoint;
//   a crease vertex with k >= 2: w sharp + (1 - w) smooth, w = min(s, 1), sharp =
//   (p_a + 6 p + p_b) / 8 for k == 2 and p for k >= 3. Exactly one crease thread writes a vertex:
//   the one whose outgoing corner at that vertex is the smallest among the vertex's creases.
// crease_inherit produces C_{l+1} in two passes (count, then fill, Sec. 3.3): each crease yields
// its two halves with sigma' = max((sigma_o + 3 sigma) / 4 - 1, 0) (the Chaikin-style rule),
// evaluated with correctly rounded FP32 operations in a fixed order; halves with sigma' = 0 are
// dropped by a scan-based compaction, which keeps the list sorted by edge id.
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
    CreaseList out;             // candidates (2 per crease)
    int *flags;
    const float *P;
    float *Pn;
    bool in4, out4;             // level l / l + 1 positions in padded float4 rows
    int *status;
};

__device__ __forceinline__ float lookup(const CreaseList &C, int K, int e) {
    int lo = 0, hi = K - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int m = __ldg(C.edge + mid);
        if (m == e) return __ldg(C.sig + mid);
        if (m < e) lo = mid + 1;
        else hi = mid - 1;
    }
    return 0.f;
}

struct EndInfo {
    int k;          // incident creases
    float S;        // their sharpness sum, in ring order from the start corner
    int n1, n2;     // the first two crease neighbours
    float s1, s2;
    int minc;       // smallest outgoing crease corner at the vertex
};

template <class Acc>
__device__ EndInfo analyse(const Acc &A, const CreaseList &C, int K, int start, int *status) {
    EndInfo r;
    r.k = 0; r.S = 0.f; r.n1 = r.n2 = -1; r.s1 = r.s2 = 0.f; r.minc = 0x7fffffff;
    int y = start, steps = 0;
    do {
        float sy = lookup(C, K, A.edge(y));
        if (sy > 0.f) {
            int nb = A.vtx(A.next(y));
            if (r.k == 0) { r.n1 = nb; r.s1 = sy; }
            else if (r.k == 1) { r.n2 = nb; r.s2 = sy; }
            r.k++;
            r.S += sy;
            r.minc = min(r.minc, y);
        }
        y = A.twin(A.prev(y));
        steps++;
    } while (y != start && steps < kMaxValence);
    if (y != start) set_status(status, ALSUB_ERR_UNSUPPORTED);
    return r;
}

__device__ __forceinline__ float chaikin(float so, float s) {
    float t = __fmul_rn(3.0f, s);
    float u = __fadd_rn(so, t);
    float w = __fmul_rn(u, 0.25f);
    float y = __fsub_rn(w, 1.0f);
    return y > 0.f ? y : 0.f;
}

template <class Acc>
__global__ void k_crease_fix(Acc A, CreaseArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (failed(a.status)) return;
    const int K = *a.in.count;
    if (i >= K) return;
    int e = a.in.edge[i], o = a.in.own[i];
    float s = a.in.sig[i];
    int t = A.twin(o);
    int va = A.vtx(o), vb = A.vtx(t);
    float3 pa = ldpv(a.P, va, a.in4), pb = ldpv(a.P, vb, a.in4);
    float3 mid = 0.5f * (pa + pb);
    int idx = a.epbase + e;
    if (s >= 1.0f) stpv(a.Pn, idx, mid, a.out4);
    else stpv(a.Pn, idx, (1.0f - s) * ldpv_rw(a.Pn, idx, a.out4) + s * mid, a.out4);
    int starts[2] = {o, t};
    int verts[2] = {va, vb};
    for (int h = 0; h < 2; h++) {
        EndInfo r = analyse(A, a.in, K, starts[h], a.status);
        if (r.minc != starts[h] || r.k < 2) continue;
        int v = verts[h];
        float sv = r.S / (float)r.k;
        float w = sv < 1.0f ? sv : 1.0f;
        float3 p = ldpv(a.P, v, a.in4);
        float3 sharp = r.k == 2 ? 0.125f * (ldpv(a.P, r.n1, a.in4) + 6.0f * p + ldpv(a.P, r.n2, a.in4)) : p;
        stpv(a.Pn, v, w * sharp + (1.0f - w) * ldpv_rw(a.Pn, v, a.out4), a.out4);
    }
}

__device__ __forceinline__ int child_corner(int x, int tri) {
    if (!tri) return 4 * x;                 // Catmull-Clark: corner 0 of child quad x
    int r = x / 3, j = x - 3 * r;           // Loop: corner 0 of child j of triangle r
    return 3 * (4 * r + j);
}

template <class Acc>
__global__ void k_crease_inherit(Acc A, CreaseArgs a, int cap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    const int K = failed(a.status) ? 0 : *a.in.count;
    if (i >= K) { a.flags[2 * i] = 0; a.flags[2 * i + 1] = 0; return; }
    int e = a.in.edge[i], o = a.in.own[i];
    float s = a.in.sig[i];
    int t = A.twin(o);
    int va = A.vtx(o), vb = A.vtx(t);
    EndInfo ra = analyse(A, a.in, K, o, a.status);
    EndInfo rb = analyse(A, a.in, K, t, a.status);
    float oa = s, ob = s;
    if (ra.k == 2) { float x = ra.n1 == vb ? ra.s2 : ra.s1; if (isfinite(x)) oa = x; }
    if (rb.k == 2) { float x = rb.n1 == va ? rb.s2 : rb.s1; if (isfinite(x)) ob = x; }
    float ca = chaikin(oa, s), cb = chaikin(ob, s);
    int ep = a.epbase + e;
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
    a.flags[2 * i] = ca > 0.f;
    a.flags[2 * i + 1] = cb > 0.f;
}

__global__ void k_crease_compact(int n, const int *__restrict__ flags, const int *__restrict__ pos,
                                 CreaseList src, CreaseList dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    int k = pos[i];
    dst.edge[k] = src.edge[i];
    dst.own[k] = src.own[i];
    dst.sig[k] = src.sig[i];
    dst.verts[2 * k] = src.verts[2 * i];
    dst.verts[2 * k + 1] = src.verts[2 * i + 1];
}

template <class F>
void with_acc(TopoImpl &T, int l, F f) {
    LevelBuf &A = T.L[l];
    if (l == 0) {
        AccL0 acc;
        acc.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0};
        f(acc);
    } else if (T.scheme == ALSUB_CATMULL_CLARK) {
        f(AccQuad{A.fv, A.tw, A.ce});
    } else {
        f(AccTri{A.fv, A.tw, A.ce});
    }
}

CreaseArgs base_args(TopoImpl &T, int l) {
    LevelBuf &A = T.L[l];
    CreaseArgs a;
    a.epbase = (int)(T.scheme == ALSUB_CATMULL_CLARK ? A.V + A.F : A.V);
    a.child_tri = T.scheme == ALSUB_LOOP;
    a.in = A.cr;
    a.out = T.ctmp;
    a.flags = T.flags;
    a.P = nullptr; a.Pn = nullptr;
    a.status = T.status;
    a.in4 = l > 0;
    a.out4 = l + 1 < T.levels;
    return a;
}

}  // namespace

void crease_fix(TopoImpl &T, int l, const float *P, float *Pn, cudaStream_t s) {
    if (T.scheme == ALSUB_SQRT3 || T.L[l].cr.cap == 0) return;
    CreaseArgs a = base_args(T, l);
    a.P = P; a.Pn = Pn;
    unsigned g = grid_for(T.L[l].cr.cap);
    with_acc(T, l, [&](auto acc) { k_crease_fix<<<g, kBlock, 0, s>>>(acc, a); });
    T.launches += 1;
}

void crease_inherit(TopoImpl &T, int l, cudaStream_t s) {
    if (T.scheme == ALSUB_SQRT3) return;
    CreaseList &dst = T.L[l + 1].cr;
    if (dst.cap == 0 || T.L[l].cr.cap == 0) {
        if (dst.count) cudaMemsetAsync(dst.count, 0, sizeof(int), s);
        return;
    }
    CreaseArgs a = base_args(T, l);
    int cap = (int)T.L[l].cr.cap;
    with_acc(T, l, [&](auto acc) { k_crease_inherit<<<grid_for(cap), kBlock, 0, s>>>(acc, a, cap); });
    scan_exclusive(T.flags, T.pos, 2LL * cap, dst.count, nullptr, T.scan_tmp, s);
    k_crease_compact<<<grid_for(2LL * cap), kBlock, 0, s>>>(2 * cap, T.flags, T.pos, T.ctmp, dst);
    T.launches += 5;
}

}  // namespace alsub
