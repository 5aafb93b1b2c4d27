// Level-0 adjacency of an arbitrary closed polygon mesh, built entirely on the device (the paper's
// point: no serial preprocessing).
//
//  * face order c = M^T 1 (Eq. fo) and the cyclic next / previous corner (the circulant action
//    maps Q_c, Q_c^{c-1} of Eq. CC_E, evaluated on demand);
//  * the twin of every corner: the corner b -> a of corner a -> b, i.e. the face-adjacency matrix F
//    (Eq. F) stored per corner, found through an open-addressing table of directed edges (the
//    symbolic pass of the implicit mapped SpGEMM of Sec. 4.2 done as one hash join: every corner
//    inserts its directed edge, every corner looks up the reverse one);
//  * the edge numbering: a corner owns its edge when its start vertex is the smaller endpoint
//    (the upper triangle of E, Eq. CC_E), or when it has no twin (a boundary edge, the entries
//    of value 1 in E that Sec. 3.2 "Boundaries" identifies); an exclusive scan over the owner
//    flags numbers the edges deterministically;
//  * for an open Catmull-Clark or Loop mesh, the list of boundary corners with each one's successor
//    along its boundary loop (the input of the boundary repair step, Fig. module_boundary);
//  * the level-0 crease list (C of Sec. 3.3) sorted by edge id.
// Non-manifold input is reported through the handle's status word, never by trapping.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ unsigned long long dir_key(int a, int b) {
    return ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
}
__device__ __forceinline__ unsigned dir_slot(unsigned long long k, unsigned mask) {
    k ^= k >> 33;                       // 64-bit finaliser (multiply-xorshift)
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (unsigned)k & mask;
}
// Returns false when the directed edge is already in the table (a duplicate: non-manifold).
__device__ bool dir_insert(const DirTable &t, int a, int b, int x) {
    const unsigned long long k = dir_key(a, b);
    unsigned h = dir_slot(k, t.mask);
    for (unsigned probe = 0; probe <= t.mask; probe++) {
        const unsigned long long old = atomicCAS(t.key + h, kEmptyKey, k);
        if (old == kEmptyKey) {
            t.val[h] = x;
            return true;
        }
        if (old == k) return false;
        h = (h + 1) & t.mask;
    }
    return false;
}
__device__ int dir_find(const DirTable &t, int a, int b) {
    const unsigned long long k = dir_key(a, b);
    unsigned h = dir_slot(k, t.mask);
    for (unsigned probe = 0; probe <= t.mask; probe++) {
        const unsigned long long q = __ldg(t.key + h);
        if (q == k) return __ldg(t.val + h);
        if (q == kEmptyKey) return -1;
        h = (h + 1) & t.mask;
    }
    return -1;
}

// Start of a level-0 build: the status word (from the mesh's device checks), the vertex degrees
// and designated corners, and the directed-edge table cleared in one pass.
__global__ void k_clear0(int V, DirTable tab, int *status, const int *mstatus, int *deg, unsigned *vc) {
    pdl_wait();
    pdl_trigger();
    const long long n = (long long)tab.mask + 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n || i < V; i += stride) {
        if (i < n) tab.key[i] = kEmptyKey;
        if (i < V) {
            deg[i] = 0;
            vc[i] = ~0u;
        }
        if (i == 0) *status = mstatus ? *mstatus : 0;    // the mesh's own device checks
    }
}

// Corner maps, vertex degrees (M 1), each vertex's smallest outgoing corner, and the directed
// edge of every corner into the table.
__global__ void k_faces(int F, const int *__restrict__ off, const int *__restrict__ fv, int *cf,
                        int *nx, int *pv, int *deg, unsigned *vc, DirTable tab, int *status) {
    pdl_wait();
    pdl_trigger();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    const int s = off[r], c = off[r + 1] - s;
    int v = fv[s];
    const int v0 = v;
    for (int j = 0; j < c; j++) {
        const int x = s + j, w = j + 1 == c ? v0 : fv[x + 1];
        cf[x] = r;
        nx[x] = s + (j + 1 == c ? 0 : j + 1);
        pv[x] = s + (j == 0 ? c - 1 : j - 1);
        atomicAdd(deg + v, 1);
        atomicMin(vc + v, (unsigned)x);
        if (!dir_insert(tab, v, w, x)) set_status(status, ALSUB_ERR_NONMANIFOLD);  // a duplicate
        v = w;
    }
}

// Twin of a -> b: the corner of b -> a (none: an open edge, i.e. a boundary: twin -1 when the
// scheme has boundary rules, else an error). A corner owns its edge when a < b or it has no
// twin; each block also counts its owner corners (the edge numbering scans the counts).
__global__ void __launch_bounds__(kBlock) k_twin(int nnz, const int *__restrict__ fv, const int *__restrict__ nx,
                                                 DirTable tab, bool open, int *tw, int *own, int *bcount,
                                                 int *status) {
    __shared__ int wsum[kBlock / 32];
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    int o = 0;
    if (x < nnz) {
        const int a = fv[x], b = fv[nx[x]];
        const int t = dir_find(tab, b, a);
        if (t < 0 && !open) set_status(status, ALSUB_ERR_UNSUPPORTED);
        tw[x] = t < 0 ? (open ? -1 : x) : t;
        o = (a < b || (t < 0 && open)) ? 1 : 0;
        own[x] = o;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int sum = 0;
        for (int w = 0; w < kBlock / 32; w++) sum += wsum[w];
        bcount[blockIdx.x] = sum;
    }
}

// Edge id of every owner corner: its block's offset (the scan of the block counts) plus its rank
// among the block's owner corners (ballots), so the numbering is the owner corners in corner order.
__global__ void __launch_bounds__(kBlock) k_eid(int nnz, const int *__restrict__ own, const int *__restrict__ boff,
                                                int *eid) {
    __shared__ int wpre[kBlock / 32];
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int o = x < nnz ? own[x] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, o);
    if (lane == 0) wpre[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < w; q++) before += wpre[q];
    if (o) eid[x] = boff[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
}

// Validation of each vertex: it is in some face, its valence is supported, and its corners form a
// single fan. Interior vertex: the ring walk x <- twin(prev(x)) returns to the start after
// exactly deg(v) steps. Boundary vertex (the walk meets a corner without twin): the walk forward
// from the start to the fan's end plus the walk backward x <- next(twin(x)) to its beginning
// visit deg(v) corners (a second fan would be missed by both).
// With `rec` (Catmull-Clark), the walk also fills the ring record of the designated corner (the
// corners in walk order, for the steps of levels >= 2 that read the vertex's ring).
__global__ void k_vertex(int V, const int *__restrict__ deg, const unsigned *__restrict__ vc,
                         const int *__restrict__ rn, const int *__restrict__ tw, const int *__restrict__ nx,
                         int *rec, int *status) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int d = deg[v];
    if (d == 0) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    if (d > kMaxValence) { set_status(status, ALSUB_ERR_UNSUPPORTED); return; }
    if (failed(status)) return;
    const int m = (int)vc[v];
    int *r = rec ? rec + (size_t)kRecInts * m : nullptr;
    int x = m, steps = 0;
    do {
        if (r && steps < kRecMaxRing) r[kRecRing + steps] = x;
        x = rn[x];
        steps++;
    } while (x >= 0 && x != m && steps <= d);
    const bool closed = x == m;
    if (x < 0) {
        int y = m;
        while (tw[y] >= 0 && steps <= d) { y = nx[tw[y]]; steps++; }
    }
    if (steps != d) set_status(status, ALSUB_ERR_NONMANIFOLD);
    if (r) r[kRecVertex] = !closed ? kRecOpen : (steps <= kRecMaxRing && steps == d ? steps : kRecLong);
}

// Boundary corners of an open mesh (twin -1), appended in any order: entry i holds the corner's
// start vertex and edge id; bidx maps the corner back to its entry.
__global__ void k_bnd0(int nnz, const int *__restrict__ fv, const int *__restrict__ tw, const int *__restrict__ ce,
                       int B, int *count, int *A, int *E, int *S, int *bidx) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz || tw[x] >= 0) return;
    const int i = atomicAdd(count, 1);
    if (i >= B) return;
    A[i] = fv[x];
    E[i] = ce[x];
    S[i] = x;                      // the corner, until k_bnd0_link replaces it
    bidx[x] = i;
}

// Successor of entry i along its loop: the boundary corner leaving the end vertex b of corner
// x = a -> b. The fan of b is walked from next(x) with y <- next(twin(y)) until the corner
// without twin (Sec. 3.2 "Boundaries": the boundary neighbours of a vertex).
__global__ void k_bnd0_link(int B, const int *__restrict__ count, const int *__restrict__ tw,
                            const int *__restrict__ nx, const int *__restrict__ bidx, int *S, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && *count != B) set_status(status, ALSUB_ERR_NONMANIFOLD);
    if (i >= B || i >= *count) return;
    const int x = S[i];
    int y = nx[x], steps = 0;
    while (tw[y] >= 0 && steps < kMaxValence) { y = nx[tw[y]]; steps++; }
    if (tw[y] >= 0) { set_status(status, ALSUB_ERR_UNSUPPORTED); S[i] = i; return; }
    const int j = bidx[y];
    S[i] = (j >= 0 && j < B) ? j : i;
}

// Boundary scan of a Catmull-Clark control mesh at creation: every face inserts its directed
// edges, then every corner whose reverse edge is missing is a boundary corner (counted) and its
// endpoints are boundary vertices (flagged), and a crease touching a boundary vertex is flagged.
__global__ void k_mb_insert(int F, const int *__restrict__ off, const int *__restrict__ fv, DirTable tab) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    const int s = off ? off[r] : 4 * r, c = off ? off[r + 1] - s : 4;
    for (int j = 0; j < c; j++) dir_insert(tab, fv[s + j], fv[s + (j + 1 == c ? 0 : j + 1)], s + j);
}
__global__ void k_mb_count(int F, const int *__restrict__ off, const int *__restrict__ fv, DirTable tab,
                           int *bv, int *out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    const int s = off ? off[r] : 4 * r, c = off ? off[r + 1] - s : 4;
    for (int j = 0; j < c; j++) {
        const int a = fv[s + j], b = fv[s + (j + 1 == c ? 0 : j + 1)];
        if (dir_find(tab, b, a) < 0) {
            atomicAdd(out, 1);
            bv[a] = 1;
            bv[b] = 1;
        }
    }
}
__global__ void k_mb_crease(int K, const int *__restrict__ cv, const int *__restrict__ bv, int *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K && (bv[cv[2 * i]] || bv[cv[2 * i + 1]])) out[1] = 1;
}
// The scan's verdict against the boundary edge count a caller stated, into the mesh's status word.
__global__ void k_mb_check(const int *__restrict__ out, long long nnz, long long B, int *mstatus) {
    const long long b = out[0];
    int st = 0;
    if (out[1]) st = ALSUB_ERR_UNSUPPORTED;                  // a crease touches a boundary vertex
    else if ((nnz + b) % 2) st = ALSUB_ERR_NONMANIFOLD;      // a directed edge repeats
    else if (b != B) st = ALSUB_ERR_INVALID_ARG;             // not the stated count
    *mstatus = st;
}

// Edge ids (an owner's own, else its twin's), owner corner of each edge, and the ring step
// twin(prev(x)).
// With `rec` (Catmull-Clark), also the edge and face parts of the corner's ring record (its
// vertex part is set to 0 here and filled by k_vertex at the designated corners).
__global__ void k_edges(int nnz, const int *__restrict__ own, const int *__restrict__ eid,
                        const int *__restrict__ tw, const int *__restrict__ pv, const int *__restrict__ nx,
                        const int *__restrict__ off, const int *__restrict__ cf, const int *e0count, int E0,
                        int *ce, int *eo, int *rn, int *rec, int *status) {
    pdl_wait();
    pdl_trigger();
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x == 0 && *e0count != E0) set_status(status, ALSUB_ERR_NONMANIFOLD);
    if (x >= nnz) return;
    const int o = own[x], t = tw[x];
    int e = o ? eid[x] : eid[t];
    e = min(max(e, 0), E0 - 1);
    ce[x] = e;
    if (o) eo[e] = x;
    rn[x] = tw[pv[x]];
    if (rec) {
        const int f = cf[x], s = off[f];
        int4 *r = reinterpret_cast<int4 *>(rec + (size_t)kRecInts * x);
        r[0] = make_int4(0, !o ? -1 : (t < 0 ? kRecOpen : t), (o && t >= 0) ? nx[t] : 0, nx[x]);
        r[1] = make_int4(x == s ? off[f + 1] - s : 0, 0, 0, 0);
    }
}

// Level-0 crease list, in input order (the crease matrix C of Sec. 3.3): each input crease
// (a, b, sigma) is mapped to its edge (the corner a -> b, from the directed-edge table) and owner
// corner and entered into the level's hash table. A crease that is not an edge of the mesh, or an
// edge tagged twice, is an input error.
__global__ void k_crease0(int K, const int *__restrict__ cv, const float *__restrict__ cs,
                          const int *__restrict__ fv, DirTable tab, const int *__restrict__ ce,
                          const int *__restrict__ own, const int *__restrict__ tw, CreaseList out,
                          int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *out.count = K;
    if (i >= K) return;
    out.edge[i] = 0; out.own[i] = 0; out.sig[i] = 0.f; out.verts[2 * i] = 0; out.verts[2 * i + 1] = 0;
    if (failed(status)) return;
    const int va = cv[2 * i], vb = cv[2 * i + 1];
    const int x = dir_find(tab, va, vb);
    if (x < 0) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    // x is the corner va -> vb: it owns the edge, or its twin vb -> va does
    const bool ox = own[x] != 0;
    const int o = ox ? x : tw[x], e = ce[x];
    const float s = cs[i];
    if (!crease_insert(out, e, s)) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    out.edge[i] = e;
    out.own[i] = o;
    out.sig[i] = s;
    out.verts[2 * i] = ox ? va : vb;           // the owner corner's start, then its end
    out.verts[2 * i + 1] = ox ? vb : va;
}

// sqrt(3) with feature edges, level 0 (the general path of sqrt3f.cu): the boundary corners (twin
// -1) are ranked in corner order by a scan of their flags and their twins become -1 - rank; the
// flags then also mark both corners of every infinitely sharp crease (a crease that is not an edge
// is an input error), which also enter the level's crease list; each triangle's flags become its
// feature bits.
__global__ void k_s3f_flags0(int nnz, const int *__restrict__ tw, int *flag) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < nnz) flag[x] = tw[x] < 0;
}

__global__ void k_s3f_rank0(int nnz, const int *__restrict__ pos, int *tw) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nnz) return;
    const int t = tw[x];
    if (t < 0) tw[x] = -1 - pos[x];
}

__global__ void k_s3f_crease0(int K, const int *__restrict__ cv, const float *__restrict__ cs, DirTable tab,
                              const int *__restrict__ tw, int *flag, int *xcount, int *xverts, float *xsig,
                              int *status) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *xcount = K;
    if (i >= K) return;
    const int a = cv[2 * i], b = cv[2 * i + 1];
    xverts[2 * i] = a;
    xverts[2 * i + 1] = b;
    xsig[i] = cs[i];
    const int x = dir_find(tab, a, b);
    if (x < 0) { set_status(status, ALSUB_ERR_INVALID_ARG); return; }
    flag[x] = 1;
    const int t = tw[x];
    if (t >= 0) flag[t] = 1;
}

__global__ void k_s3f_mask0(int F, const int *__restrict__ flag, unsigned char *fm) {
    pdl_wait();
    pdl_trigger();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < F) fm[q] = (unsigned char)(flag[3 * q] | flag[3 * q + 1] << 1 | flag[3 * q + 2] << 2);
}

}  // namespace

void level0_build(TopoImpl &T, cudaStream_t s) {
    MeshImpl &M = *T.mesh;
    LevelBuf &L0 = T.L[0];
    const int V = M.V, F = M.F, nnz = M.nnz, E0 = (int)L0.E;
    const long long slots = (long long)T.dir.mask + 1;
    launch_pdl(k_clear0, std::min<unsigned>(grid_for(std::max<long long>(slots, V)), 1024u), kBlock, s, V, T.dir,
               T.status, (const int *)M.d_status, T.deg, reinterpret_cast<unsigned *>(T.vc0));
    launch_pdl(k_faces, grid_for(F), kBlock, s, F, (const int *)M.d_off, (const int *)M.d_fv, T.cf0, T.nx0, T.pv0,
               T.deg, reinterpret_cast<unsigned *>(T.vc0), T.dir, T.status);
    const unsigned nb = grid_for(nnz);
    const bool open = M.scheme != ALSUB_SQRT3 || M.B > 0;  // closed sqrt(3) meshes are checked closed
    launch_pdl(k_twin, nb, kBlock, s, nnz, (const int *)M.d_fv, (const int *)T.nx0, T.dir, open, L0.tw, T.own0,
               T.flags, T.status);
    T.launches += 5 + scan_exclusive(T.flags, T.pos, nb, T.e0count, nullptr, T.scan_tmp, s);
    launch_pdl(k_eid, nb, kBlock, s, nnz, (const int *)T.own0, (const int *)T.pos, T.eid);
    launch_pdl(k_edges, grid_for(nnz), kBlock, s, nnz, (const int *)T.own0, (const int *)T.eid, (const int *)L0.tw,
               (const int *)T.pv0, (const int *)T.nx0, (const int *)M.d_off, (const int *)T.cf0,
               (const int *)T.e0count, E0, L0.ce, T.eo0, T.rn0, T.rec0, T.status);
    if (L0.B > 0 && T.levels > 0 && M.scheme != ALSUB_SQRT3) {
        // (the list exists when a step follows: levels >= 1.) The per-corner edge-id temporaries
        // are dead: they map boundary corners to entries
        cudaMemsetAsync(T.bcount, 0, sizeof(int), s);
        k_bnd0<<<grid_for(nnz), kBlock, 0, s>>>(nnz, M.d_fv, L0.tw, L0.ce, M.B, T.bcount, L0.bA, L0.bE, L0.bS,
                                                T.eid);
        k_bnd0_link<<<grid_for(M.B), kBlock, 0, s>>>(M.B, T.bcount, L0.tw, T.nx0, T.eid, L0.bS, T.status);
        T.launches += 2;
    }
}

alsub_status level_boundary_flags(int V, int F, long long n, const int *off, const int *fv, int *flag,
                                  const DevAlloc &A, cudaStream_t s) {
    int k = 4;
    while ((1LL << k) < 2 * n) k++;
    const size_t slots = (size_t)1 << k;
    char *buf = nullptr;
    if (dev_malloc(A, &buf, slots * (sizeof(unsigned long long) + sizeof(int)) + 16, s) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "boundary flags: device allocation failed");
    }
    DirTable tab;
    tab.key = (unsigned long long *)buf;
    tab.val = (int *)(buf + slots * sizeof(unsigned long long));
    tab.mask = (unsigned)(slots - 1);
    int *count = tab.val + slots;              // k_mb_count's boundary edge counter (unused here)
    cudaMemsetAsync(tab.key, 0xff, slots * sizeof(unsigned long long), s);
    cudaMemsetAsync(count, 0, sizeof(int), s);
    cudaMemsetAsync(flag, 0, sizeof(int) * (size_t)V, s);
    k_mb_insert<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, tab);
    k_mb_count<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, tab, flag, count);
    dev_free(A, buf, s);
    return ALSUB_OK;
}

namespace {

// The scan's kernels into a temporary buffer (released after them, stream-ordered); *out gets
// the device address of [boundary edges, crease at a boundary].
alsub_status boundary_scan_kernels(MeshImpl &M, cudaStream_t s, char **buf_out, int **out_dev) {
    int k = 4;
    while ((1LL << k) < 2LL * M.nnz) k++;
    const size_t slots = (size_t)1 << k;
    char *buf = nullptr;
    const size_t bytes = slots * (sizeof(unsigned long long) + sizeof(int)) + sizeof(int) * ((size_t)M.V + 2);
    if (dev_malloc(M.alloc, &buf, bytes, s) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "mesh boundary scan: device allocation failed");
    }
    DirTable tab;
    tab.key = (unsigned long long *)buf;
    tab.val = (int *)(buf + slots * sizeof(unsigned long long));
    tab.mask = (unsigned)(slots - 1);
    int *bv = tab.val + slots, *out = bv + M.V;
    cudaMemsetAsync(tab.key, 0xff, slots * sizeof(unsigned long long), s);
    cudaMemsetAsync(bv, 0, sizeof(int) * ((size_t)M.V + 2), s);
    k_mb_insert<<<grid_for(M.F), kBlock, 0, s>>>(M.F, M.d_off, M.d_fv, tab);
    k_mb_count<<<grid_for(M.F), kBlock, 0, s>>>(M.F, M.d_off, M.d_fv, tab, bv, out);
    if (M.K > 0) k_mb_crease<<<grid_for(M.K), kBlock, 0, s>>>(M.K, M.d_cv, bv, out);
    *buf_out = buf;
    *out_dev = out;
    return ALSUB_OK;
}

}  // namespace

alsub_status mesh_boundary_check(MeshImpl &M, cudaStream_t s, long long B_stated) {
    char *buf = nullptr;
    int *out = nullptr;
    alsub_status st = boundary_scan_kernels(M, s, &buf, &out);
    if (st != ALSUB_OK) return st;
    k_mb_check<<<1, 1, 0, s>>>(out, (long long)M.nnz, B_stated, M.d_status);
    dev_free(M.alloc, buf, s);
    M.B = (int)B_stated;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, "mesh boundary check failed");
}

alsub_status mesh_boundary_scan(MeshImpl &M, cudaStream_t s, long long *B, bool *crease_at_boundary) {
    *B = 0;
    *crease_at_boundary = false;
    char *buf = nullptr;
    int *out = nullptr;
    alsub_status st = boundary_scan_kernels(M, s, &buf, &out);
    if (st != ALSUB_OK) return st;
    int h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(M.alloc, buf, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return report(ALSUB_ERR_DEVICE, "mesh boundary scan failed");
    }
    *B = h[0];
    *crease_at_boundary = h[1] != 0;
    return ALSUB_OK;
}

void level0_validate(TopoImpl &T, cudaStream_t s) {
    k_vertex<<<grid_for(T.mesh->V), kBlock, 0, s>>>(T.mesh->V, T.deg, reinterpret_cast<unsigned *>(T.vc0),
                                                    T.rn0, T.L[0].tw, T.nx0, T.rec0, T.status);
    T.launches += 1;
}

void level0_creases(TopoImpl &T, cudaStream_t s) {
    if (T.scheme == ALSUB_SQRT3) return;     // sqrt(3) creases are feature flags (s3f_level0)
    MeshImpl &M = *T.mesh;
    LevelBuf &L0 = T.L[0];
    CreaseList &C = L0.cr;
    if (C.cap > 0) {
        crease_table_clear(C, s);
        k_crease0<<<grid_for(M.K), kBlock, 0, s>>>(M.K, M.d_cv, M.d_cs, M.d_fv, T.dir, L0.ce, T.own0, L0.tw,
                                                   C, T.status);
        T.launches += 1;
    } else if (C.count) {
        cudaMemsetAsync(C.count, 0, sizeof(int), s);
    }
}

void s3f_level0(TopoImpl &T, cudaStream_t s) {
    MeshImpl &M = *T.mesh;
    LevelBuf &L0 = T.L[0];
    const int nnz = M.nnz;
    launch_pdl(k_s3f_flags0, grid_for(nnz), kBlock, s, nnz, (const int *)L0.tw, T.flags);
    T.launches += 3 + scan_exclusive(T.flags, T.pos, nnz, nullptr, nullptr, T.scan_tmp, s);
    launch_pdl(k_s3f_rank0, grid_for(nnz), kBlock, s, nnz, (const int *)T.pos, L0.tw);
    if (M.K > 0) {
        launch_pdl(k_s3f_crease0, grid_for(M.K), kBlock, s, M.K, (const int *)M.d_cv, (const float *)M.d_cs, T.dir,
                   (const int *)L0.tw, T.flags, L0.cr.xcount, L0.cr.xverts, L0.cr.xsig, T.status);
        T.launches += 1;
    }
    if (L0.fm) launch_pdl(k_s3f_mask0, grid_for(M.F), kBlock, s, M.F, (const int *)T.flags, L0.fm);
}

}  // namespace alsub
