// Level-0 adjacency of an arbitrary closed polygon mesh, built entirely on the device (the paper's
// point: no serial preprocessing).
//
//  * face order c = M^T 1 (Eq. fo) and the cyclic next / previous corner (the circulant action
//    maps Q_c, Q_c^{c-1} of Eq. CC_E, evaluated on demand);
//  * the vertex -> corner incidence (a counting sort of M by row: the symbolic pass of the implicit
//    mapped SpGEMM, Sec. 4.2) and from it the twin of every corner: the corner b -> a of corner
//    a -> b, i.e. the face-adjacency matrix F (Eq. F) stored per corner;
//  * the edge numbering: a corner owns its edge when its start vertex is the smaller endpoint
//    (the upper triangle of E, Eq. CC_E); an exclusive scan over the owner flags numbers the
//    edges deterministically;
//  * the level-0 crease list (C of Sec. 3.3) sorted by edge id.
// Non-manifold input is reported through the handle's status word, never by trapping.
#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

__global__ void k_faces(int F, const int *__restrict__ off, const int *__restrict__ fv, int *cf,
                        int *nx, int *pv, int *deg) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    int s = off[r], c = off[r + 1] - s;
    for (int j = 0; j < c; j++) {
        int x = s + j;
        cf[x] = r;
        nx[x] = s + (j + 1 == c ? 0 : j + 1);
        pv[x] = s + (j == 0 ? c - 1 : j - 1);
        atomicAdd(deg + fv[x], 1);
    }
}

__global__ void k_bucket(int nnz, const int *__restrict__ fv, const int *__restrict__ voff,
                         int *vfill, int *vbk) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz) return;
    int v = fv[x];
    int pos = atomicAdd(vfill + v, 1);
    vbk[voff[v] + pos] = x;
}

// Twin of a -> b: the unique corner b -> a in b's bucket. The bucket order is not deterministic,
// but the result of the search is.
__global__ void k_twin(int nnz, const int *__restrict__ fv, const int *__restrict__ nx,
                       const int *__restrict__ voff, const int *__restrict__ vbk, int *tw, int *own,
                       int *status) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz) return;
    int a = fv[x], b = fv[nx[x]];
    int found = x, cnt = 0;
    const int qb0 = voff[b], qb1 = voff[b + 1], qa0 = voff[a], qa1 = voff[a + 1];
#pragma unroll 4
    for (int q = qb0; q < qb1; q++) {
        int d = vbk[q];
        if (fv[nx[d]] == a) { found = d; cnt++; }
    }
    if (cnt == 0) set_status(status, ALSUB_ERR_UNSUPPORTED);      // open edge: boundary
    else if (cnt > 1) set_status(status, ALSUB_ERR_NONMANIFOLD);
#pragma unroll 4
    for (int q = qa0; q < qa1; q++) {                              // duplicate directed edge
        int d = vbk[q];
        if (d != x && fv[nx[d]] == b) set_status(status, ALSUB_ERR_NONMANIFOLD);
    }
    tw[x] = cnt == 1 ? found : x;
    own[x] = a < b ? 1 : 0;
}

// Designated outgoing corner of each vertex (the smallest) and the single-fan check: the ring
// walk x <- twin(prev(x)) must return to the start after exactly deg(v) steps.
__global__ void k_vertex(int V, const int *__restrict__ voff, const int *__restrict__ vbk,
                         const int *__restrict__ tw, const int *__restrict__ pv, int *vc, int *status) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    int s = voff[v], deg = voff[v + 1] - s;
    if (deg == 0) { set_status(status, ALSUB_ERR_INVALID_ARG); vc[v] = 0; return; }
    if (deg > kMaxValence) { set_status(status, ALSUB_ERR_UNSUPPORTED); vc[v] = vbk[s]; return; }
    int m = vbk[s];
    for (int q = s + 1; q < s + deg; q++) m = min(m, vbk[q]);
    vc[v] = m;
    if (failed(status)) return;
    int x = m, steps = 0;
    do { x = tw[pv[x]]; steps++; } while (x != m && steps <= deg);
    if (steps != deg) set_status(status, ALSUB_ERR_NONMANIFOLD);
}

__global__ void k_edges(int nnz, const int *__restrict__ own, const int *__restrict__ eid,
                        const int *__restrict__ tw, const int *e0count, int E0, int *ce, int *eo,
                        int *status) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x == 0 && *e0count != E0) set_status(status, ALSUB_ERR_NONMANIFOLD);
    if (x >= nnz) return;
    int e = own[x] ? eid[x] : eid[tw[x]];
    e = min(max(e, 0), E0 - 1);
    ce[x] = e;
    if (own[x]) eo[e] = x;
}

// Level-0 crease list, in input order (the crease matrix C of Sec. 3.3): each input crease
// (a, b, sigma) is mapped to its edge and owner corner and entered into the level's hash table.
// A crease that is not an edge of the mesh, or an edge tagged twice, is an input error.
__global__ void k_crease0(int K, const int *__restrict__ cv, const float *__restrict__ cs,
                          const int *__restrict__ fv, const int *__restrict__ nx,
                          const int *__restrict__ voff, const int *__restrict__ vbk,
                          const int *__restrict__ ce, const int *__restrict__ own,
                          const int *__restrict__ tw, CreaseList out, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *out.count = K;
    if (i >= K) return;
    out.edge[i] = 0; out.own[i] = 0; out.sig[i] = 0.f; out.verts[2 * i] = 0; out.verts[2 * i + 1] = 0;
    if (failed(status)) return;
    const int a = cv[2 * i], b = cv[2 * i + 1];
    // every candidate of a's bucket is tested (no early exit), so the loads of different
    // candidates do not wait on one another; the first match is taken
    int x = -1;
    const int q0 = voff[a], q1 = voff[a + 1];
#pragma unroll 4
    for (int q = q0; q < q1; q++) {
        const int d = vbk[q];
        if (x < 0 && fv[nx[d]] == b) x = d;
    }
    if (x < 0) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    const int o = own[x] ? x : tw[x], e = ce[x];
    const float s = cs[i];
    if (!crease_insert(out, e, s)) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    out.edge[i] = e;
    out.own[i] = o;
    out.sig[i] = s;
    out.verts[2 * i] = fv[o];
    out.verts[2 * i + 1] = fv[tw[o]];
}

}  // namespace

void level0_build(TopoImpl &T, cudaStream_t s) {
    MeshImpl &M = *T.mesh;
    LevelBuf &L0 = T.L[0];
    const int V = M.V, F = M.F, nnz = M.nnz, E0 = (int)L0.E;
    cudaMemsetAsync(T.status, 0, sizeof(int), s);
    cudaMemsetAsync(T.deg, 0, sizeof(int) * (size_t)V, s);
    cudaMemsetAsync(T.vfill, 0, sizeof(int) * (size_t)V, s);
    k_faces<<<grid_for(F), kBlock, 0, s>>>(F, M.d_off, M.d_fv, T.cf0, T.nx0, T.pv0, T.deg);
    T.launches += 5 + scan_exclusive(T.deg, T.voff, V, T.voff + V, nullptr, T.scan_tmp, s);
    k_bucket<<<grid_for(nnz), kBlock, 0, s>>>(nnz, M.d_fv, T.voff, T.vfill, T.vbk);
    k_twin<<<grid_for(nnz), kBlock, 0, s>>>(nnz, M.d_fv, T.nx0, T.voff, T.vbk, L0.tw, T.own0, T.status);
    k_vertex<<<grid_for(V), kBlock, 0, s>>>(V, T.voff, T.vbk, L0.tw, T.pv0, T.vc0, T.status);
    T.launches += scan_exclusive(T.own0, T.eid, nnz, T.e0count, nullptr, T.scan_tmp, s);
    k_edges<<<grid_for(nnz), kBlock, 0, s>>>(nnz, T.own0, T.eid, L0.tw, T.e0count, E0, L0.ce, T.eo0,
                                             T.status);
}

void level0_creases(TopoImpl &T, cudaStream_t s) {
    MeshImpl &M = *T.mesh;
    LevelBuf &L0 = T.L[0];
    CreaseList &C = L0.cr;
    if (C.cap > 0) {
        crease_table_clear(C, s);
        k_crease0<<<grid_for(M.K), kBlock, 0, s>>>(M.K, M.d_cv, M.d_cs, M.d_fv, T.nx0, T.voff, T.vbk,
                                                   L0.ce, T.own0, L0.tw, C, T.status);
        T.launches += 1;
    } else if (C.count) {
        cudaMemsetAsync(C.count, 0, sizeof(int), s);
    }
}

}  // namespace alsub
