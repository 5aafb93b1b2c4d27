// Mesh reordering (Sec. 4.5): reverse Cuthill-McKee on the graph of the mesh Laplacian permutes
// the vertices (the rows of M), then the faces (the columns) are sorted by their first non-zero
// row, the least new index among their vertices.
//
// Cuthill-McKee is a breadth-first labelling: a component starts at its unlabelled vertex of least
// (degree, index); the labelled vertices are visited in label order and each labels its unlabelled
// neighbours in increasing (degree, index). The device runs it one breadth-first level at a time:
// a vertex w of the next level is labelled by the first vertex of the current level that reaches
// it, i.e. by its neighbour of least label there (atomicMin), and the next level's labels follow
// from sorting its vertices by (that parent's label, degree, index): a counting sort on the parent
// (exclusive scan of the per-parent counts) and a short insertion sort inside each parent's group
// (its size is at most the parent's degree). That is the serial order exactly, whatever order the
// atomics resolve in. Reversing the order gives RCM (George 1971). Faces are bucketed by their
// least new vertex index the same way, each bucket sorted by input face index (stable).
//
// Cost: one pass over the corners for the graph, then per breadth-first level three small kernels,
// one exclusive scan and one read-back of the level's size (the host decides when a component
// ends), plus one pass over the vertices per connected component to find its start.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

// parent word of a vertex no labelled vertex has reached yet (a byte pattern, so one memset sets
// it; labels stay below it)
constexpr int kUnreached = 0x7f7f7f7f;

// vertex degree of the Laplacian graph: count both directions of every face edge (duplicates
// removed afterwards)
__global__ void k_rcm_pair_count(int F, const int *__restrict__ off, const int *__restrict__ fv, int *acnt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int s = __ldg(off + f), c = __ldg(off + f + 1) - s;
    for (int j = 0; j < c; j++) {
        const int u = __ldg(fv + s + j), w = __ldg(fv + s + (j + 1 == c ? 0 : j + 1));
        if (u == w) continue;
        atomicAdd(acnt + u, 1);
        atomicAdd(acnt + w, 1);
    }
}

__global__ void k_rcm_pair_fill(int F, const int *__restrict__ off, const int *__restrict__ fv,
                                const int *__restrict__ aoff, int *afill, int *adj) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int s = __ldg(off + f), c = __ldg(off + f + 1) - s;
    for (int j = 0; j < c; j++) {
        const int u = __ldg(fv + s + j), w = __ldg(fv + s + (j + 1 == c ? 0 : j + 1));
        if (u == w) continue;
        adj[aoff[u] + atomicAdd(afill + u, 1)] = w;
        adj[aoff[w] + atomicAdd(afill + w, 1)] = u;
    }
}

// in-place heapsort of a[0 .. n) (ascending)
__device__ void heap_sift(int *a, int i, int n) {
    const int x = a[i];
    for (;;) {
        int c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && a[c + 1] > a[c]) c++;
        if (a[c] <= x) break;
        a[i] = a[c];
        i = c;
    }
    a[i] = x;
}

__device__ void heap_sort(int *a, int n) {
    for (int i = n / 2 - 1; i >= 0; i--) heap_sift(a, i, n);
    for (int m = n - 1; m > 0; m--) {
        const int t = a[0]; a[0] = a[m]; a[m] = t;
        heap_sift(a, 0, m);
    }
}

// each vertex's neighbour list sorted and its repeats dropped (in place): deg[v] distinct
// neighbours at adj[aoff[v] ..]
__global__ void k_rcm_unique(int V, const int *__restrict__ aoff, int *adj, int *deg) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    int *a = adj + aoff[v];
    const int n = aoff[v + 1] - aoff[v];
    heap_sort(a, n);
    int d = 0;
    for (int i = 0; i < n; i++)
        if (d == 0 || a[i] != a[d - 1]) a[d++] = a[i];
    deg[v] = d;
}

// the least (degree, index) among the unlabelled vertices
__global__ void k_rcm_seed_min(int V, const int *__restrict__ label, const int *__restrict__ deg,
                               unsigned long long *key) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long k = ~0ull;
    if (v < V && label[v] < 0) k = ((unsigned long long)(unsigned)deg[v] << 32) | (unsigned)v;
    for (int o = 16; o > 0; o >>= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
    if ((threadIdx.x & 31) == 0 && k != ~0ull) atomicMin(key, k);
}

__global__ void k_rcm_seed_set(const unsigned long long *key, int at, int *label, int *order) {
    const int v = (int)(unsigned)(*key & 0xffffffffull);
    label[v] = at;
    order[at] = v;
}

// vertices order[lo .. hi) (the current level) reach their unlabelled neighbours: each keeps its
// least parent label; the first to reach it appends it to the candidate list
__global__ void k_rcm_expand(int lo, int hi, const int *__restrict__ order, const int *__restrict__ aoff,
                             const int *__restrict__ adj, const int *__restrict__ deg,
                             const int *__restrict__ label, int *parent, int *cand, int *ncand) {
    const int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= hi) return;
    const int u = order[k];
    const int *a = adj + aoff[u];
    const int d = deg[u];
    for (int i = 0; i < d; i++) {
        const int w = a[i];
        if (label[w] >= 0) continue;
        if (atomicMin(parent + w, k) == kUnreached) cand[atomicAdd(ncand, 1)] = w;
    }
}

__global__ void k_rcm_group_count(int n, int lo, const int *__restrict__ cand, const int *__restrict__ parent,
                                  int *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(cnt + (parent[cand[i]] - lo), 1);
}

// candidates into their parent's group (in any order inside it); cnt counts down to 0
__global__ void k_rcm_group_place(int n, int lo, int hi, const int *__restrict__ cand,
                                  const int *__restrict__ parent, const int *__restrict__ start, int *cnt,
                                  int *order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int w = cand[i], g = parent[w] - lo;
    order[hi + start[g] + atomicSub(cnt + g, 1) - 1] = w;
}

// each parent's group sorted by (degree, index); the group's vertices take their labels
__global__ void k_rcm_group_sort(int width, int hi, int n, const int *__restrict__ start,
                                 const int *__restrict__ deg, int *order, int *label) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= width) return;
    const int b = hi + start[g], e = hi + (g + 1 < width ? start[g + 1] : n);
    for (int i = b + 1; i < e; i++) {
        const int w = order[i];
        const long long kw = ((long long)deg[w] << 32) | (unsigned)w;
        int j = i - 1;
        while (j >= b) {
            const int x = order[j];
            if ((((long long)deg[x] << 32) | (unsigned)x) <= kw) break;
            order[j + 1] = x;
            j--;
        }
        order[j + 1] = w;
    }
    for (int i = b; i < e; i++) label[order[i]] = i;
}

// RCM: new index V-1-label; vmap[new] = old
__global__ void k_rcm_vmap(int V, const int *__restrict__ order, int *newid, int *vmap) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V) return;
    const int v = order[k];
    newid[v] = V - 1 - k;
    vmap[V - 1 - k] = v;
}

// faces bucketed by their least new vertex index
__global__ void k_rcm_face_key(int F, const int *__restrict__ off, const int *__restrict__ fv,
                               const int *__restrict__ newid, int *fkey, int *fcnt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int s = __ldg(off + f), c = __ldg(off + f + 1) - s;
    int m = INT_MAX;
    for (int j = 0; j < c; j++) m = min(m, newid[__ldg(fv + s + j)]);
    fkey[f] = m;
    atomicAdd(fcnt + m, 1);
}

__global__ void k_rcm_face_place(int F, const int *__restrict__ fkey, const int *__restrict__ fstart, int *fcnt,
                                 int *fmap) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int k = fkey[f];
    fmap[fstart[k] + atomicSub(fcnt + k, 1) - 1] = f;
}

// each bucket in input face order; new face sizes
__global__ void k_rcm_face_sort(int V, int F, const int *__restrict__ fstart, const int *__restrict__ off,
                                int *fmap, int *fsize) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int b = fstart[v], e = v + 1 < V ? fstart[v + 1] : F;
    for (int i = b + 1; i < e; i++) {
        const int f = fmap[i];
        int j = i - 1;
        while (j >= b && fmap[j] > f) {
            fmap[j + 1] = fmap[j];
            j--;
        }
        fmap[j + 1] = f;
    }
    for (int i = b; i < e; i++) fsize[i] = __ldg(off + fmap[i] + 1) - __ldg(off + fmap[i]);
}

__global__ void k_rcm_face_fill(int F, const int *__restrict__ fmap, const int *__restrict__ off,
                                const int *__restrict__ fv, const int *__restrict__ newid,
                                const int *__restrict__ noff, int *nfv) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int g = fmap[f], s = __ldg(off + g), c = __ldg(off + g + 1) - s, t = noff[f];
    for (int j = 0; j < c; j++) nfv[t + j] = newid[__ldg(fv + s + j)];
}

__global__ void k_rcm_creases(int K, const int *__restrict__ cv, const int *__restrict__ newid, int *ncv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * K) ncv[i] = newid[cv[i]];
}

}  // namespace

alsub_status reorder_mesh(const MeshImpl &M, cudaStream_t s, MeshImpl &out, int *levels_out) {
    const int V = M.V, F = M.F;
    const long long nnz = M.nnz;
    if (V < 1 || F < 1) return report(ALSUB_ERR_INVALID_ARG, "reorder: empty mesh");
    if (2 * nnz > INT_MAX || V >= kUnreached)
        return report(ALSUB_ERR_UNSUPPORTED, "reorder: more than 2^30 corners or 0x7f7f7f7f vertices");
    // temporaries: acnt / aoff (V + 1), afill, deg, label, parent, order, cand, cnt, start, newid (V);
    // adj (2 nnz); fkey, fsize (F); a seed key
    const size_t nV = (size_t)V + 1, nF = (size_t)F;
    const long long nmax = std::max<long long>({(long long)V + 1, (long long)F});
    const size_t stmp = scan_tmp_bytes(nmax);
    const size_t ints = 10 * nV + 2 * (size_t)nnz + 2 * nF + 8;
    char *buf = nullptr;
    const DevAlloc &DA = M.alloc;             // the reordered mesh takes the source mesh's allocator
    out.alloc = DA;
    if (dev_malloc(DA, &buf, 4 * ints + stmp + 512, s) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "reorder: device allocation failed");
    }
    int *aoff = (int *)buf, *afill = aoff + nV, *deg = afill + nV, *label = deg + nV, *parent = label + nV;
    int *order = parent + nV, *cand = order + nV, *cnt = cand + nV, *start = cnt + nV, *newid = start + nV;
    int *adj = newid + nV, *fkey = adj + 2 * (size_t)nnz, *fsize = fkey + nF, *tot = fsize + nF;
    unsigned long long *seed = (unsigned long long *)(((uintptr_t)(tot + 8) + 15) & ~(uintptr_t)15);
    void *tmp = (void *)(((uintptr_t)(seed + 2) + 255) & ~(uintptr_t)255);
    auto bail = [&](alsub_status st, const char *what) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        dev_free(DA, buf, s);
        return report(st, what);
    };

    // graph of the Laplacian: adjacency lists, sorted, without repeats
    cudaMemsetAsync(afill, 0, 4 * nV, s);
    cudaMemsetAsync(tot, 0, 4 * 8, s);
    k_rcm_pair_count<<<grid_for(F), kBlock, 0, s>>>(F, M.d_off, M.d_fv, afill);
    scan_exclusive(afill, aoff, V + 1, nullptr, nullptr, tmp, s);
    cudaMemsetAsync(afill, 0, 4 * nV, s);
    k_rcm_pair_fill<<<grid_for(F), kBlock, 0, s>>>(F, M.d_off, M.d_fv, aoff, afill, adj);
    k_rcm_unique<<<grid_for(V), kBlock, 0, s>>>(V, aoff, adj, deg);
    cudaMemsetAsync(label, 0xff, 4 * nV, s);          // -1: unlabelled
    cudaMemsetAsync(parent, 0x7f, 4 * nV, s);         // kUnreached
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bail(ALSUB_ERR_DEVICE, cudaGetErrorString(e));

    int hi = 0, levels = 0;
    while (hi < V) {
        // a new component: its start vertex
        cudaMemsetAsync(seed, 0xff, sizeof(unsigned long long), s);
        k_rcm_seed_min<<<grid_for(V), kBlock, 0, s>>>(V, label, deg, seed);
        k_rcm_seed_set<<<1, 1, 0, s>>>(seed, hi, label, order);
        int lo = hi;
        hi = lo + 1;
        for (;;) {
            const int width = hi - lo;
            cudaMemsetAsync(tot, 0, sizeof(int), s);
            k_rcm_expand<<<grid_for(width), kBlock, 0, s>>>(lo, hi, order, aoff, adj, deg, label, parent, cand, tot);
            int n = 0;
            e = cudaMemcpyAsync(&n, tot, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return bail(ALSUB_ERR_DEVICE, "reorder: breadth-first step failed");
            levels++;
            if (n == 0) break;
            if (n > V - hi) return bail(ALSUB_ERR_DEVICE, "reorder: breadth-first level overflows");
            cudaMemsetAsync(cnt, 0, 4 * (size_t)width, s);
            k_rcm_group_count<<<grid_for(n), kBlock, 0, s>>>(n, lo, cand, parent, cnt);
            scan_exclusive(cnt, start, width, nullptr, nullptr, tmp, s);
            k_rcm_group_place<<<grid_for(n), kBlock, 0, s>>>(n, lo, hi, cand, parent, start, cnt, order);
            k_rcm_group_sort<<<grid_for(width), kBlock, 0, s>>>(width, hi, n, start, deg, order, label);
            lo = hi;
            hi += n;
        }
    }
    if (levels_out) *levels_out = levels;

    out.scheme = M.scheme;
    out.V = V; out.F = F; out.nnz = (int)nnz; out.K = M.K; out.B = M.B;
    out.sigma_max = M.sigma_max;
    out.stream = s;
    e = dev_malloc(DA, &out.d_off, sizeof(int) * (size_t)(F + 1), s);
    if (e == cudaSuccess) e = dev_malloc(DA, &out.d_fv, sizeof(int) * (size_t)nnz, s);
    if (e == cudaSuccess) e = dev_malloc(DA, &out.d_vmap, sizeof(int) * (size_t)V, s);
    if (e == cudaSuccess) e = dev_malloc(DA, &out.d_fmap, sizeof(int) * (size_t)F, s);
    if (e == cudaSuccess && M.K) e = dev_malloc(DA, &out.d_cv, sizeof(int) * 2 * (size_t)M.K, s);
    if (e == cudaSuccess && M.K) e = dev_malloc(DA, &out.d_cs, sizeof(float) * (size_t)M.K, s);
    if (e != cudaSuccess) return bail(ALSUB_ERR_OOM, "reorder: device allocation failed");
    k_rcm_vmap<<<grid_for(V), kBlock, 0, s>>>(V, order, newid, out.d_vmap);
    cudaMemsetAsync(cnt, 0, 4 * nV, s);
    k_rcm_face_key<<<grid_for(F), kBlock, 0, s>>>(F, M.d_off, M.d_fv, newid, fkey, cnt);
    scan_exclusive(cnt, start, V, nullptr, nullptr, tmp, s);
    k_rcm_face_place<<<grid_for(F), kBlock, 0, s>>>(F, fkey, start, cnt, out.d_fmap);
    k_rcm_face_sort<<<grid_for(V), kBlock, 0, s>>>(V, F, start, M.d_off, out.d_fmap, fsize);
    scan_exclusive(fsize, out.d_off, F, out.d_off + F, nullptr, tmp, s);
    k_rcm_face_fill<<<grid_for(F), kBlock, 0, s>>>(F, out.d_fmap, M.d_off, M.d_fv, newid, out.d_off, out.d_fv);
    if (M.K) {
        k_rcm_creases<<<grid_for(2 * M.K), kBlock, 0, s>>>(M.K, M.d_cv, newid, out.d_cv);
        cudaMemcpyAsync(out.d_cs, M.d_cs, sizeof(float) * (size_t)M.K, cudaMemcpyDeviceToDevice, s);
    }
    dev_free(DA, buf, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
    return ALSUB_OK;
}

}  // namespace alsub
