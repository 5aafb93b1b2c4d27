// Matrix-free adjoint of a Catmull-Clark refinement step on a closed mesh: g_l = R_l^T g_{l+1}
// as a gather per coarse vertex, without atomics and without storing R_l or its transpose.
//
// R_l's rows are the step's stencils (Sec. 3.2, Eq. 2 and Eq. pos_update, the crease rules of
// Sec. 3.3):
//   face point   f_r = (1/c) sum of r's corners;
//   edge point   (1 - s) (p_a + p_b + f_r + f_t) / 4 + s (p_a + p_b) / 2, s = min(sigma, 1);
//   vertex point (1 - w) [(1 - 2/n) p + 1/n^2 sum p_j + 1/n^2 sum f_j] + w q, with w = min(S/k, 1)
//                for k >= 2 incident creases (else 0) and q = (p_n1 + 6 p + p_n2) / 8 (k = 2) or p.
// The column of coarse vertex v collects, face by face around v (face r at v's corner y, order c):
//   f_r                          1/c
//   the edge y -> next (v, u)    (1 - s)(1/4 + 1/(4c) + 1/(4c')) + s/2     (c': the face across)
//   the vertex point of u        a_u (1 + 1/c + 1/c') + (sigma > 0 ? b_u : 0)
//   each far edge of r           (1 - s) / (4c)
//   each far vertex w of r       a_w / c
// plus its own vertex point with weight g_v, where per vertex a = (1 - w)/n^2, b = w/8 when k = 2
// (else 0) and g = (1 - w)(1 - 2/n + sum_j 1/(n^2 c_j)) + w (3/4 when k = 2, 1 when k >= 3). Each
// edge at v is the edge y -> next of exactly one face around v, so nothing is counted twice; a
// vertex or edge that two faces around v share (a valence-2 vertex) is counted once per face, as
// its stencil counts it. The per-vertex (a, b, g), each vertex's designated corner, the slot each
// corner's contribution goes to and each creased edge's min(sigma, 1) depend on the topology only:
// they are computed once per level when the operator is built.
// Each level runs in two passes: per coarse face, the terms above that the face contributes at each
// of its corners (one float4 per corner, the face's own rows read coalesced; on levels >= 1 a
// valence-4 vertex's four contributions land side by side); then per coarse vertex, its own term
// plus its contributions.
#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

// Level 0: polygons (corner maps of Level0). Levels >= 1: quads, corner 4r + k.
template <bool L0>
struct AdjTopo {
    Level0 z;
    const int *fv, *tw, *ce;    // the level's (stored) face table, twins and edge ids
    int l;
    __device__ int face(int y) const { return L0 ? __ldg(z.cf + y) : y >> 2; }
    __device__ int first(int r) const { return L0 ? __ldg(z.off + r) : 4 * r; }
    __device__ int order(int r) const { return L0 ? __ldg(z.off + r + 1) - __ldg(z.off + r) : 4; }
    __device__ int ring(int y) const { return L0 ? __ldg(z.rn + y) : __ldg(tw + quad_prev(y)); }
    __device__ bool designated(int x) const {
        return L0 ? __ldg(z.vc + __ldg(z.fv + x)) == x : cc_vown(l, x, z);
    }
};

struct AdjArgs {
    int V, F;                 // coarse counts: level l + 1 numbers [old V | face points F | edge points]
    const float *G;           // gradient of level l + 1
    float *g;                 // gradient of level l
    bool G4, g4;              // float4 rows (intermediate levels) or packed xyz
    const float4 *coef;       // (a, b, g, 0) per coarse vertex
    const int *corner;        // each coarse vertex's designated corner
    const int *pidx;          // levels >= 1: where corner x's contribution goes (4 v + i for the i-th
                              // ring corner of a valence-4 vertex v, else 4 V + x)
    const float *sh;          // min(sigma, 1) per coarse edge (when CREASED)
    int *status;
};

template <bool CREASED>
__device__ __forceinline__ float sharp(const CreaseList &C, int e) {
    return CREASED ? crease_lookup(C, e) : 0.f;
}
// the clamped sharpness min(sigma, 1) of a coarse edge (0: smooth)
template <bool CREASED>
__device__ __forceinline__ float edge_s(const AdjArgs &a, int e) {
    return CREASED ? __ldg(a.sh + e) : 0.f;
}

// Per-vertex coefficients (a, b, g) of one level and each vertex's designated corner, from one
// ring walk per designated corner.
template <bool L0, bool CREASED>
__global__ void __launch_bounds__(kBlock) k_adj_coef(AdjTopo<L0> A, int nnz, int V, CreaseList cr, float4 *coef,
                                                     int *corner, int *pidx, int *status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz || failed(status) || !A.designated(x)) return;
    const int v = __ldg(A.fv + x);
    corner[v] = x;
    int y = x, n = 0, k = 0;
    int rc[4] = {-1, -1, -1, -1};
    float S = 0.f, invc = 0.f;
    do {
        if (n < 4) rc[n] = y;
        invc += 1.0f / (float)A.order(A.face(y));
        const float sg = sharp<CREASED>(cr, __ldg(A.ce + y));
        if (sg > 0.f) { k++; S += sg; }
        y = A.ring(y);
        n++;
    } while (y >= 0 && y != x && n < kMaxValence);
    if (y != x) { set_status(status, ALSUB_ERR_UNSUPPORTED); return; }   // open or too long
    if (pidx) {
        // the contributions of a valence-4 vertex's ring faces go to four adjacent slots
        if (n == 4) {
            for (int i = 0; i < 4; i++) pidx[rc[i]] = 4 * v + i;
        } else {
            int z = x, m = 0;
            do { pidx[z] = 4 * V + z; z = A.ring(z); m++; } while (z >= 0 && z != x && m < kMaxValence);
        }
    }
    const float inv = 1.0f / (float)n;
    float w = 0.f;
    if (k >= 2) { w = S / (float)k; w = w < 1.0f ? w : 1.0f; }
    const float a = (1.0f - w) * inv * inv;
    const float b = k == 2 ? 0.125f * w : 0.f;
    const float q = k == 2 ? 0.75f : (k >= 3 ? 1.0f : 0.f);
    const float gm = (1.0f - w) * (1.0f - 2.0f * inv + inv * inv * invc) + w * q;
    coef[v] = make_float4(a, b, gm, (float)n);
}

// min(sigma, 1) of every edge of a creased level (the hash table's lookups, done once).
__global__ void k_adj_sharp(int E, CreaseList cr, float *sh) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const float s = crease_lookup(cr, e);
    sh[e] = s < 1.0f ? s : 1.0f;
}

// Levels >= 1 (quads), two passes. k_adj_face: per coarse face r, the whole contribution of r
// to the vertex at each corner k (the terms of the column sum above that belong to face r at that
// corner), written to part[pidx[4r + k]]; its rows are its own (coalesced) and the 17 values it
// gathers are independent of one another. k_adj_vert: per coarse vertex, its own vertex-point term
// plus its contributions (a valence-4 vertex reads them as 64 contiguous bytes).
template <bool CREASED>
__global__ void __launch_bounds__(kBlock) k_adj_face(const int *__restrict__ fv, const int *__restrict__ ce,
                                                     AdjArgs a, float4 *__restrict__ part) {
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.F || failed(a.status)) return;
    const int VF = a.V + a.F;
    const int4 vr = ld4(fv + 4 * (size_t)r), er = ld4(ce + 4 * (size_t)r), pr = ld4(a.pidx + 4 * (size_t)r);
    const int vv[4] = {vr.x, vr.y, vr.z, vr.w}, ee[4] = {er.x, er.y, er.z, er.w};
    float3 gv[4], ge[4];
    float4 cf[4];
    float sk[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        gv[k] = ldpv(a.G, vv[k], a.G4);
        ge[k] = ldpv(a.G, VF + ee[k], a.G4);
        cf[k] = __ldg(a.coef + vv[k]);
        sk[k] = edge_s<CREASED>(a, ee[k]);
    }
    const float3 gf = 0.25f * ldpv(a.G, a.V + r, a.G4);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int k1 = (k + 1) & 3, k2 = (k + 2) & 3;
        float3 p = gf;
        p += ((1.0f - sk[k]) * 0.375f + 0.5f * sk[k]) * ge[k];                    // ring edge v_k v_k+1
        p += (1.5f * cf[k1].x + (sk[k] > 0.f ? cf[k1].y : 0.f)) * gv[k1];          // its end vertex
        p += ((1.0f - sk[k1]) * 0.0625f) * ge[k1];                                  // the far edges
        p += ((1.0f - sk[k2]) * 0.0625f) * ge[k2];
        p += (0.25f * cf[k2].x) * gv[k2];                                           // the far vertex
        part[comp(pr, k)] = make_float4(p.x, p.y, p.z, 0.f);
    }
}

// Level 0: the same first pass over polygons, one thread per corner x of face r (order c, corners
// s .. s + c - 1; c' of the face across x's edge read through the twin).
template <bool CREASED>
__global__ void __launch_bounds__(kBlock) k_adj_face0(AdjTopo<true> A, AdjArgs a, int nnz, float4 *__restrict__ part) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz || failed(a.status)) return;
    const int VF = a.V + a.F;
    const int r = A.face(x), s0 = A.first(r), c = A.order(r), k = x - s0;
    const float ic = 1.0f / (float)c;
    const float3 gf = ic * ldpv(a.G, a.V + r, a.G4);
    {
        const int t = __ldg(A.tw + x);
        const float ict = 1.0f / (float)A.order(A.face(t));
        const int e0 = __ldg(A.ce + x);
        const float s0c = edge_s<CREASED>(a, e0);
        float3 p = gf;
        p += ((1.0f - s0c) * (0.25f + 0.25f * (ic + ict)) + 0.5f * s0c) * ldpv(a.G, VF + e0, a.G4);
        const int u = __ldg(A.fv + s0 + (k + 1 == c ? 0 : k + 1));
        const float4 cu = __ldg(a.coef + u);
        p += (cu.x * (1.0f + ic + ict) + (s0c > 0.f ? cu.y : 0.f)) * ldpv(a.G, u, a.G4);
        for (int q = 1; q + 1 < c; q++) {
            const int yq = s0 + (k + q) % c;
            const int eq = __ldg(A.ce + yq);
            p += ((1.0f - edge_s<CREASED>(a, eq)) * 0.25f * ic) * ldpv(a.G, VF + eq, a.G4);
            if (q >= 2) {
                const int w = __ldg(A.fv + yq);
                p += (__ldg(a.coef + w).x * ic) * ldpv(a.G, w, a.G4);
            }
        }
        part[x] = make_float4(p.x, p.y, p.z, 0.f);
    }
}

template <bool L0>
__global__ void __launch_bounds__(kBlock) k_adj_vert(AdjTopo<L0> A, AdjArgs a, const float4 *__restrict__ part) {
    pdl_wait();
    pdl_trigger();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V || failed(a.status)) return;
    const float4 cv = __ldg(a.coef + v);
    float3 acc = cv.z * ldpv(a.G, v, a.G4);
    if (!L0 && cv.w == 4.0f) {
        // a valence-4 vertex: its four contributions side by side
        const float4 *q = part + 4 * (size_t)v;
        const float4 p0 = __ldg(q), p1 = __ldg(q + 1), p2 = __ldg(q + 2), p3 = __ldg(q + 3);
        acc += f3(p0.x, p0.y, p0.z);
        acc += f3(p1.x, p1.y, p1.z);
        acc += f3(p2.x, p2.y, p2.z);
        acc += f3(p3.x, p3.y, p3.z);
    } else {
        const int x = __ldg(a.corner + v);
        const size_t off = L0 ? 0 : 4 * (size_t)a.V;    // levels >= 1: after the valence-4 slots
        int y = x, n = 0;
        do {
            const float4 p = __ldg(part + off + y);
            acc += f3(p.x, p.y, p.z);
            y = A.ring(y);
            n++;
        } while (y >= 0 && y != x && n < kMaxValence);
        if (y != x) set_status(a.status, ALSUB_ERR_UNSUPPORTED);
    }
    stpv(a.g, v, acc, a.g4);
}

template <bool L0>
AdjTopo<L0> adj_topo(const TopoImpl &T, int l) {
    AdjTopo<L0> A;
    A.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0, T.rn0};
    const LevelBuf &B = T.L[l];
    A.fv = l == 0 ? T.mesh->d_fv : B.fv;
    A.tw = B.tw;
    A.ce = B.ce;
    A.l = l;
    return A;
}

bool level_creased(const TopoImpl &T, int l) { return l <= T.levels && T.L[l].cr.cap > 0; }

}  // namespace

bool adjoint_supported(const TopoImpl &T) {
    return T.scheme == ALSUB_CATMULL_CLARK && T.mesh->B == 0 && T.levels > 0;
}

bool adjoint_level_creased(const TopoImpl &T, int l) { return level_creased(T, l); }

void adjoint_prepare(TopoImpl &T, int l, const AdjLevel &P, cudaStream_t s) {
    const int nnz = (int)T.L[l].nnz, V = (int)T.L[l].V;
    const unsigned g = grid_for(nnz);
    const CreaseList &C = T.L[l].cr;
    const bool cr = level_creased(T, l);
    // every vertex of a closed manifold level has exactly one designated corner; the zero fill
    // keeps every entry a valid corner regardless
    cudaMemsetAsync(P.corner, 0, sizeof(int) * (size_t)T.L[l].V, s);
    if (P.pidx) cudaMemsetAsync(P.pidx, 0, sizeof(int) * (size_t)nnz, s);   // every slot in bounds
    if (l == 0) {
        if (cr) k_adj_coef<true, true><<<g, kBlock, 0, s>>>(adj_topo<true>(T, l), nnz, V, C, P.coef, P.corner, P.pidx, T.status);
        else k_adj_coef<true, false><<<g, kBlock, 0, s>>>(adj_topo<true>(T, l), nnz, V, C, P.coef, P.corner, P.pidx, T.status);
    } else {
        if (cr) k_adj_coef<false, true><<<g, kBlock, 0, s>>>(adj_topo<false>(T, l), nnz, V, C, P.coef, P.corner, P.pidx, T.status);
        else k_adj_coef<false, false><<<g, kBlock, 0, s>>>(adj_topo<false>(T, l), nnz, V, C, P.coef, P.corner, P.pidx, T.status);
    }
    if (cr) k_adj_sharp<<<grid_for(T.L[l].E), kBlock, 0, s>>>((int)T.L[l].E, C, P.sh);
    T.launches += cr ? 2 : 1;
}

void adjoint_step(TopoImpl &T, int l, const float *G, bool G4, float *g, bool g4, const AdjLevel &P,
                  float4 *part, cudaStream_t s) {
    AdjArgs a;
    a.V = (int)T.L[l].V;
    a.F = (int)T.L[l].F;
    a.G = G; a.G4 = G4;
    a.g = g; a.g4 = g4;
    a.coef = P.coef;
    a.corner = P.corner;
    a.pidx = P.pidx;
    a.sh = P.sh;
    a.status = T.status;
    const bool cr = level_creased(T, l);
    if (l == 0) {
        const int n0 = (int)T.L[0].nnz;
        if (cr) launch_pdl(k_adj_face0<true>, grid_for(n0), kBlock, s, adj_topo<true>(T, l), a, n0, part);
        else launch_pdl(k_adj_face0<false>, grid_for(n0), kBlock, s, adj_topo<true>(T, l), a, n0, part);
        launch_pdl(k_adj_vert<true>, grid_for(a.V), kBlock, s, adj_topo<true>(T, l), a, (const float4 *)part);
    } else {
        const LevelBuf &B = T.L[l];
        if (cr) launch_pdl(k_adj_face<true>, grid_for(a.F), kBlock, s, (const int *)B.fv, (const int *)B.ce, a, part);
        else launch_pdl(k_adj_face<false>, grid_for(a.F), kBlock, s, (const int *)B.fv, (const int *)B.ce, a, part);
        launch_pdl(k_adj_vert<false>, grid_for(a.V), kBlock, s, adj_topo<false>(T, l), a, (const float4 *)part);
    }
    T.launches += 2;
}

}  // namespace alsub
