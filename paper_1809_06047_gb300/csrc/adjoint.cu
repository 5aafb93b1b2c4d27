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
// its stencil counts it. The per-vertex (a, b, g) depend on the topology only: they are computed
// once per level when the operator is built.
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
    int nnz;                  // corners of the coarse level
    int V, F;                 // coarse counts: level l + 1 numbers [old V | face points F | edge points]
    const float *G;           // gradient of level l + 1
    float *g;                 // gradient of level l
    bool G4, g4;              // float4 rows (intermediate levels) or packed xyz
    const float4 *coef;       // (a, b, g, 0) per coarse vertex
    const int *corner;        // each coarse vertex's designated corner
    const int4 *ring;         // levels >= 1: a valence-4 vertex's ring corners (x = -1: another valence)
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
__global__ void __launch_bounds__(kBlock) k_adj_coef(AdjTopo<L0> A, int nnz, CreaseList cr, float4 *coef,
                                                     int *corner, int4 *ring, int *status) {
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
    if (ring) ring[v] = n == 4 ? make_int4(rc[0], rc[1], rc[2], rc[3]) : make_int4(-1, -1, -1, -1);
    const float inv = 1.0f / (float)n;
    float w = 0.f;
    if (k >= 2) { w = S / (float)k; w = w < 1.0f ? w : 1.0f; }
    const float a = (1.0f - w) * inv * inv;
    const float b = k == 2 ? 0.125f * w : 0.f;
    const float q = k == 2 ? 0.75f : (k >= 3 ? 1.0f : 0.f);
    const float gm = (1.0f - w) * (1.0f - 2.0f * inv + inv * inv * invc) + w * q;
    coef[v] = make_float4(a, b, gm, 0.f);
}

// min(sigma, 1) of every edge of a creased level (the hash table's lookups, done once).
__global__ void k_adj_sharp(int E, CreaseList cr, float *sh) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const float s = crease_lookup(cr, e);
    sh[e] = s < 1.0f ? s : 1.0f;
}

// The column sum of one coarse vertex (its designated corner x).
template <bool L0, bool CREASED>
__device__ __forceinline__ void adj_vertex(const AdjTopo<L0> &A, const AdjArgs &a, int x) {
    const int v = __ldg(A.fv + x);
    const int VF = a.V + a.F;
    float3 acc = __ldg(a.coef + v).z * ldpv(a.G, v, a.G4);
    int y = x, n = 0;
    do {
        const int r = A.face(y), s0 = A.first(r), c = A.order(r), j = y - s0;
        const float ic = 1.0f / (float)c;
        acc += ic * ldpv(a.G, a.V + r, a.G4);                          // the face point
        // the edge y -> next and the vertex at its end
        const int t = __ldg(A.tw + y);
        const float ict = L0 ? 1.0f / (float)A.order(A.face(t)) : 0.25f;
        const int e0 = __ldg(A.ce + y);
        const float s0c = edge_s<CREASED>(a, e0);
        acc += ((1.0f - s0c) * (0.25f + 0.25f * (ic + ict)) + 0.5f * s0c) * ldpv(a.G, VF + e0, a.G4);
        const int yn = s0 + (j + 1 == c ? 0 : j + 1);
        const int u = __ldg(A.fv + yn);
        const float4 cu = __ldg(a.coef + u);
        acc += (cu.x * (1.0f + ic + ict) + (s0c > 0.f ? cu.y : 0.f)) * ldpv(a.G, u, a.G4);
        // the far edges (from next to prev) and the far vertices (strictly between them)
        for (int q = 1; q + 1 < c; q++) {
            const int yq = s0 + (j + q) % c;
            const int eq = __ldg(A.ce + yq);
            const float sqc = edge_s<CREASED>(a, eq);
            acc += ((1.0f - sqc) * 0.25f * ic) * ldpv(a.G, VF + eq, a.G4);
            if (q >= 2) {
                const int w = __ldg(A.fv + yq);
                acc += (__ldg(a.coef + w).x * ic) * ldpv(a.G, w, a.G4);
            }
        }
        y = A.ring(y);
        n++;
    } while (y >= 0 && y != x && n < kMaxValence);
    stpv(a.g, v, acc, a.g4);
}

// Levels >= 1 (quads): the ring is taken four faces per round, first the chain of twins (the only
// dependent loads), then the rows of the four faces, then every gradient and coefficient they
// name, so a valence-4 vertex waits for six round trips instead of three per face.
template <bool CREASED>
__device__ __forceinline__ void adj_vertex_quads(const AdjTopo<false> &A, const AdjArgs &a, int v) {
    const int VF = a.V + a.F;
    const int4 rc = __ldg(a.ring + v);               // a valence-4 vertex: its four ring corners
    const int x = rc.x >= 0 ? rc.x : __ldg(a.corner + v);
    float3 acc = __ldg(a.coef + v).z * ldpv(a.G, v, a.G4);
    int y = x, n = 0;
    bool done = false, first = true;
    while (!done && n < kMaxValence) {
        int ys[4];
        bool use[4];
        if (first && rc.x >= 0) {
            ys[0] = rc.x; ys[1] = rc.y; ys[2] = rc.z; ys[3] = rc.w;
            use[0] = use[1] = use[2] = use[3] = true;
            y = x;
            n = 4;
            done = true;
        } else {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                use[q] = !done;
                ys[q] = y;
                if (!done) {
                    y = A.ring(y);
                    n++;
                    done = y == x || y < 0 || n >= kMaxValence;
                }
            }
        }
        first = false;
        int4 fr[4], er[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = use[q] ? ys[q] >> 2 : 0;
            fr[q] = use[q] ? ld4(A.fv + 4 * (size_t)r) : make_int4(0, 0, 0, 0);
            er[q] = use[q] ? ld4(A.ce + 4 * (size_t)r) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (!use[q]) continue;
            const int r = ys[q] >> 2, j = ys[q] & 3, j1 = (j + 1) & 3, j2 = (j + 2) & 3;
            const int u = comp(fr[q], j1), w = comp(fr[q], j2);
            const int e0 = comp(er[q], j), e1 = comp(er[q], j1), e2 = comp(er[q], j2);
            const float s0c = edge_s<CREASED>(a, e0), s1c = edge_s<CREASED>(a, e1), s2c = edge_s<CREASED>(a, e2);
            const float4 cu = __ldg(a.coef + u), cw = __ldg(a.coef + w);
            acc += 0.25f * ldpv(a.G, a.V + r, a.G4);
            acc += ((1.0f - s0c) * 0.375f + 0.5f * s0c) * ldpv(a.G, VF + e0, a.G4);
            acc += (1.5f * cu.x + (s0c > 0.f ? cu.y : 0.f)) * ldpv(a.G, u, a.G4);
            acc += ((1.0f - s1c) * 0.0625f) * ldpv(a.G, VF + e1, a.G4);
            acc += ((1.0f - s2c) * 0.0625f) * ldpv(a.G, VF + e2, a.G4);
            acc += (0.25f * cw.x) * ldpv(a.G, w, a.G4);
        }
    }
    if (y != x) set_status(a.status, ALSUB_ERR_UNSUPPORTED);
    stpv(a.g, v, acc, a.g4);
}

// One thread per coarse vertex, from the designated corner the build recorded.
template <bool L0, bool CREASED>
__global__ void __launch_bounds__(kBlock) k_adj_gather(AdjTopo<L0> A, AdjArgs a) {
    pdl_wait();
    pdl_trigger();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V || failed(a.status)) return;
    if constexpr (L0) adj_vertex<true, CREASED>(A, a, __ldg(a.corner + v));
    else adj_vertex_quads<CREASED>(A, a, v);
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
    const int nnz = (int)T.L[l].nnz;
    const unsigned g = grid_for(nnz);
    const CreaseList &C = T.L[l].cr;
    const bool cr = level_creased(T, l);
    // every vertex of a closed manifold level has exactly one designated corner; the zero fill
    // keeps every entry a valid corner regardless
    cudaMemsetAsync(P.corner, 0, sizeof(int) * (size_t)T.L[l].V, s);
    if (P.ring) cudaMemsetAsync(P.ring, 0xff, sizeof(int4) * (size_t)T.L[l].V, s);   // -1: walk
    if (l == 0) {
        if (cr) k_adj_coef<true, true><<<g, kBlock, 0, s>>>(adj_topo<true>(T, l), nnz, C, P.coef, P.corner, P.ring, T.status);
        else k_adj_coef<true, false><<<g, kBlock, 0, s>>>(adj_topo<true>(T, l), nnz, C, P.coef, P.corner, P.ring, T.status);
    } else {
        if (cr) k_adj_coef<false, true><<<g, kBlock, 0, s>>>(adj_topo<false>(T, l), nnz, C, P.coef, P.corner, P.ring, T.status);
        else k_adj_coef<false, false><<<g, kBlock, 0, s>>>(adj_topo<false>(T, l), nnz, C, P.coef, P.corner, P.ring, T.status);
    }
    if (cr) k_adj_sharp<<<grid_for(T.L[l].E), kBlock, 0, s>>>((int)T.L[l].E, C, P.sh);
    T.launches += cr ? 2 : 1;
}

void adjoint_step(TopoImpl &T, int l, const float *G, bool G4, float *g, bool g4, const AdjLevel &P,
                  cudaStream_t s) {
    AdjArgs a;
    a.nnz = (int)T.L[l].nnz;
    a.V = (int)T.L[l].V;
    a.F = (int)T.L[l].F;
    a.G = G; a.G4 = G4;
    a.g = g; a.g4 = g4;
    a.coef = P.coef;
    a.corner = P.corner;
    a.ring = P.ring;
    a.sh = P.sh;
    a.status = T.status;
    const bool cr = level_creased(T, l);
    const unsigned grid = grid_for(a.V);
    if (l == 0) {
        if (cr) launch_pdl(k_adj_gather<true, true>, grid, kBlock, s, adj_topo<true>(T, l), a);
        else launch_pdl(k_adj_gather<true, false>, grid, kBlock, s, adj_topo<true>(T, l), a);
    } else {
        if (cr) launch_pdl(k_adj_gather<false, true>, grid, kBlock, s, adj_topo<false>(T, l), a);
        else launch_pdl(k_adj_gather<false, false>, grid, kBlock, s, adj_topo<false>(T, l), a);
    }
    T.launches += 1;
}

}  // namespace alsub
