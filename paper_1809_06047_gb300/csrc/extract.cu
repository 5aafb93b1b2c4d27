// Selective subdivision (Sec. 3.4, Fig. module_selective): the extraction matrices X_i (rows of the
// identity: the kept vertices) and X-ring_i (columns of the identity: the kept faces) built on the
// device from a level of a Catmull-Clark or Loop topology, and the extracted mesh
// M' = X_i M X-ring_i with its positions P' = X_i P.
//
// Selection: x_0 = the given vertex mask, or the extraordinary vertices (valence != 4 for
// Catmull-Clark, != 6 for Loop, Eq. vo, of vertices on no boundary edge) and the ends of the
// level's live creases. Propagation, `rings`
// times: q_i = M^T x_i (faces with a selected vertex), x_{i+1} = M q_i (the vertices of those
// faces). Where the region touches itself at a vertex only (two fans of kept faces), every face
// around that vertex is kept too, until no such vertex is left, so the result is a manifold. Kept
// faces and vertices keep their relative order (exclusive scans over the flags), so the
// extraction is deterministic. A crease is kept when every face around both its ends is kept.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

// face r's corners: [off[r], off[r+1]) or, for a uniform quad level (off == nullptr), [4r, 4r+4)
__device__ __forceinline__ void face_range(const int *off, int r, int &s, int &c) {
    if (off) { s = __ldg(off + r); c = __ldg(off + r + 1) - s; }
    else { s = 4 * r; c = 4; }
}

__global__ void k_x_iota(int n, int step, int *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = step * i;
}

__global__ void k_x_valence(int F, const int *__restrict__ off, const int *__restrict__ fv, int *deg) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    int s, c;
    face_range(off, r, s, c);
    for (int j = 0; j < c; j++) atomicAdd(deg + __ldg(fv + s + j), 1);
}

// default selection: interior extraordinary vertices (bnd: 1 on a boundary edge)
__global__ void k_x_select(int V, const int *__restrict__ deg, const int *__restrict__ bnd, int regular,
                           int *x) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V) x[v] = (deg[v] != regular && !bnd[v]) ? 1 : 0;
}
__global__ void k_x_select_mask(int V, const unsigned char *__restrict__ mask, int *x) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V) x[v] = mask[v] ? 1 : 0;
}
__global__ void k_x_select_creases(const int *__restrict__ count, int cap, const int *__restrict__ cv,
                                   const float *__restrict__ cs, int *x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap || i >= *count || !(cs[i] > 0.f)) return;
    x[cv[2 * i]] = 1;
    x[cv[2 * i + 1]] = 1;
}

// q = M^T x: a face is kept when one of its vertices is selected
__global__ void k_x_faces(int F, const int *__restrict__ off, const int *__restrict__ fv, const int *__restrict__ x,
                          int *q, int *ord) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    int s, c;
    face_range(off, r, s, c);
    int hit = 0;
    for (int j = 0; j < c; j++) hit |= __ldg(x + __ldg(fv + s + j));
    q[r] = hit ? 1 : 0;
    ord[r] = hit ? c : 0;
}
// x = M q: the vertices of the kept faces (every writer stores 1: no race on the value); with cnt,
// also the number of kept faces around each vertex
__global__ void k_x_verts(int F, const int *__restrict__ off, const int *__restrict__ fv, const int *__restrict__ q,
                          int *x, int *cnt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F || !q[r]) return;
    int s, c;
    face_range(off, r, s, c);
    for (int j = 0; j < c; j++) {
        const int v = __ldg(fv + s + j);
        x[v] = 1;
        if (cnt) atomicAdd(cnt + v, 1);
    }
}

// Pinches: a vertex with two or more boundary edges of the region leaving it (as many fans of kept
// faces) takes all its faces. Directed edges of the kept faces into a table, then per kept corner
// whose reverse edge is missing one more outgoing boundary edge at its start vertex.
__device__ __forceinline__ unsigned long long x_key(int a, int b) {
    return ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
}
__device__ __forceinline__ unsigned x_slot(unsigned long long k, unsigned mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (unsigned)k & mask;
}
__global__ void k_x_edges(int F, const int *__restrict__ off, const int *__restrict__ fv, const int *__restrict__ q,
                          unsigned long long *key, unsigned mask) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F || !q[r]) return;
    int s, c;
    face_range(off, r, s, c);
    for (int j = 0; j < c; j++) {
        const unsigned long long k = x_key(__ldg(fv + s + j), __ldg(fv + s + (j + 1 == c ? 0 : j + 1)));
        unsigned h = x_slot(k, mask);
        for (unsigned p = 0; p <= mask; p++) {
            const unsigned long long old = atomicCAS(key + h, ~0ull, k);
            if (old == ~0ull || old == k) break;
            h = (h + 1) & mask;
        }
    }
}
__global__ void k_x_outb(int F, const int *__restrict__ off, const int *__restrict__ fv, const int *__restrict__ q,
                         const unsigned long long *__restrict__ key, unsigned mask, int *outb) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F || !q[r]) return;
    int s, c;
    face_range(off, r, s, c);
    for (int j = 0; j < c; j++) {
        const int a = __ldg(fv + s + j), b = __ldg(fv + s + (j + 1 == c ? 0 : j + 1));
        const unsigned long long k = x_key(b, a);
        unsigned h = x_slot(k, mask);
        bool found = false;
        for (unsigned p = 0; p <= mask; p++) {
            const unsigned long long cur = key[h];
            if (cur == k) { found = true; break; }
            if (cur == ~0ull) break;
            h = (h + 1) & mask;
        }
        if (!found) atomicAdd(outb + a, 1);
    }
}
__global__ void k_x_pinch(int V, const int *__restrict__ outb, int *x, int *count) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int p = outb[v] >= 2 ? 1 : 0;
    x[v] = p;
    if (p) atomicAdd(count, 1);
}
__global__ void k_x_faces_or(int F, const int *__restrict__ off, const int *__restrict__ fv, const int *__restrict__ x,
                             int *q) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F || q[r]) return;
    int s, c;
    face_range(off, r, s, c);
    int hit = 0;
    for (int j = 0; j < c; j++) hit |= __ldg(x + __ldg(fv + s + j));
    if (hit) q[r] = 1;
}
__global__ void k_x_orders(int F, const int *__restrict__ off, const int *__restrict__ q, int *ord) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    int s, c;
    face_range(off, r, s, c);
    ord[r] = q[r] ? c : 0;
}

// the kept creases: live, both ends with every face around them kept
__global__ void k_x_crease_flags(const int *__restrict__ count, int cap, const int *__restrict__ cv,
                                 const float *__restrict__ cs, const int *__restrict__ cnt,
                                 const int *__restrict__ deg, int *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    int f = 0;
    if (i < *count && cs[i] > 0.f) {
        const int a = cv[2 * i], b = cv[2 * i + 1];
        f = (cnt[a] == deg[a] && cnt[b] == deg[b]) ? 1 : 0;
    }
    flag[i] = f;
}

__global__ void k_x_fill_faces(int F, const int *__restrict__ off, const int *__restrict__ fv, const int *__restrict__ q,
                               const int *__restrict__ fpos, const int *__restrict__ noff,
                               const int *__restrict__ vpos, int *off_out, int *fv_out, int *fmap) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F || !q[r]) return;
    int s, c;
    face_range(off, r, s, c);
    const int f = fpos[r], o = noff[r];
    off_out[f] = o;
    fmap[f] = r;
    for (int j = 0; j < c; j++) fv_out[o + j] = vpos[__ldg(fv + s + j)];
}
__global__ void k_x_fill_verts(int V, const int *__restrict__ x, const int *__restrict__ vpos, int *vmap) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V && x[v]) vmap[vpos[v]] = v;
}
__global__ void k_x_fill_creases(int cap, const int *__restrict__ flag, const int *__restrict__ cpos,
                                 const int *__restrict__ cv, const float *__restrict__ cs,
                                 const int *__restrict__ vpos, int *cv_out, float *cs_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap || !flag[i]) return;
    const int k = cpos[i];
    cv_out[2 * k] = vpos[cv[2 * i]];
    cv_out[2 * k + 1] = vpos[cv[2 * i + 1]];
    cs_out[k] = cs[i];
}

__global__ void k_x_gather(int n, const int *__restrict__ vmap, const float *__restrict__ P, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = __ldg(vmap + i);
    out[3 * (size_t)i + 0] = __ldg(P + 3 * (size_t)v + 0);
    out[3 * (size_t)i + 1] = __ldg(P + 3 * (size_t)v + 1);
    out[3 * (size_t)i + 2] = __ldg(P + 3 * (size_t)v + 2);
}

}  // namespace

alsub_status extract_level(TopoImpl &T, int level, const unsigned char *mask, int rings, cudaStream_t s,
                           MeshImpl &out) {
    const LevelBuf &L = T.L[level];
    const int V = (int)L.V, F = (int)L.F;
    const int *off = level == 0 ? T.mesh->d_off : nullptr;   // refined Catmull-Clark: quads
    const bool tri = level > 0 && T.scheme != ALSUB_CATMULL_CLARK;  // refined Loop: offsets 3r
    const int *fv = L.fv;
    // live creases of the level (exported: endpoints and sharpness, count on the device)
    const CreaseList &C = L.cr;
    int cap = 0;
    if (C.cap > 0) {
        T.launches += crease_export(T, level, s);
        cap = (int)C.cap;
    }
    // temporaries: deg, x, bnd, cnt, vpos (V); q, ord, fpos, noff (F); flags, cpos (cap); totals
    const size_t nV = (size_t)V, nF = (size_t)F, nC = (size_t)std::max(cap, 1);
    const long long nmax = std::max<long long>({(long long)V, (long long)F, (long long)nC});
    const size_t stmp = scan_tmp_bytes(nmax);
    const size_t ints = 5 * nV + 4 * nF + 2 * nC + 8 + (tri ? nF + 1 : 0);
    char *buf = nullptr;
    const DevAlloc &DA = T.alloc;       // the extracted mesh takes the source mesh's allocator
    out.alloc = DA;
    if (dev_malloc(DA, &buf, 4 * ints + stmp + 256, s) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "extraction: device allocation failed");
    }
    int *deg = (int *)buf, *x = deg + nV, *bnd = x + nV, *cnt = bnd + nV, *vpos = cnt + nV;
    int *q = vpos + nV, *ord = q + nF, *fpos = ord + nF, *noff = fpos + nF;
    int *flag = noff + nF, *cpos = flag + nC, *tot = cpos + nC, *toff = tot + 8;
    void *tmp = (void *)(((uintptr_t)(toff + (tri ? nF + 1 : 0)) + 255) & ~(uintptr_t)255);
    if (tri) {
        k_x_iota<<<grid_for(F + 1), kBlock, 0, s>>>(F + 1, 3, toff);
        off = toff;
    }
    cudaMemsetAsync(deg, 0, 4 * nV, s);
    cudaMemsetAsync(bnd, 0, 4 * nV, s);
    cudaMemsetAsync(cnt, 0, 4 * nV, s);
    cudaMemsetAsync(tot, 0, 4 * 8, s);            // 0..3 totals, 4 pinch count
    k_x_valence<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, deg);
    if (mask) {
        k_x_select_mask<<<grid_for(V), kBlock, 0, s>>>(V, mask, x);
    } else {
        alsub_status st = level_boundary_flags(V, F, L.nnz, off, fv, bnd, DA, s);
        if (st != ALSUB_OK) {
            dev_free(DA, buf, s);
            return st;
        }
        k_x_select<<<grid_for(V), kBlock, 0, s>>>(V, deg, bnd, T.scheme == ALSUB_CATMULL_CLARK ? 4 : 6, x);
        if (cap) k_x_select_creases<<<grid_for(cap), kBlock, 0, s>>>(C.xcount, cap, C.xverts, C.xsig, x);
    }
    for (int i = 0; i < rings; i++) {
        k_x_faces<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, x, q, ord);
        if (i + 1 < rings) {
            cudaMemsetAsync(x, 0, 4 * nV, s);
            k_x_verts<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, q, x, nullptr);
        }
    }
    // pinches, until none is left (each round only adds faces)
    {
        int k = 4;
        while ((1LL << k) < 2 * L.nnz) k++;
        const size_t slots = (size_t)1 << k;
        unsigned long long *key = nullptr;
        if (dev_malloc(DA, &key, slots * sizeof(unsigned long long), s) != cudaSuccess) {
            dev_free(DA, buf, s);
            return report(ALSUB_ERR_OOM, "extraction: device allocation failed");
        }
        bool clean = false;
        for (int round = 0; round < 64 && !clean; round++) {
            cudaMemsetAsync(key, 0xff, slots * sizeof(unsigned long long), s);
            cudaMemsetAsync(cnt, 0, 4 * nV, s);                  // outgoing boundary edges, for now
            cudaMemsetAsync(tot + 4, 0, sizeof(int), s);
            k_x_edges<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, q, key, (unsigned)(slots - 1));
            k_x_outb<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, q, key, (unsigned)(slots - 1), cnt);
            k_x_pinch<<<grid_for(V), kBlock, 0, s>>>(V, cnt, x, tot + 4);
            int pinches = 0;
            cudaError_t e = cudaMemcpyAsync(&pinches, tot + 4, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                dev_free(DA, key, s);
                dev_free(DA, buf, s);
                return report(ALSUB_ERR_DEVICE, "extraction failed");
            }
            clean = pinches == 0;
            if (!clean) k_x_faces_or<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, x, q);
        }
        dev_free(DA, key, s);
        if (!clean) {
            dev_free(DA, buf, s);
            return report(ALSUB_ERR_UNSUPPORTED, "extraction: the region still touches itself after 64 rounds");
        }
    }
    k_x_orders<<<grid_for(F), kBlock, 0, s>>>(F, off, q, ord);
    cudaMemsetAsync(x, 0, 4 * nV, s);
    cudaMemsetAsync(cnt, 0, 4 * nV, s);
    k_x_verts<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, q, x, cnt);
    scan_exclusive(q, fpos, F, tot + 0, nullptr, tmp, s);
    scan_exclusive(ord, noff, F, tot + 1, nullptr, tmp, s);
    scan_exclusive(x, vpos, V, tot + 2, nullptr, tmp, s);
    if (cap) {
        k_x_crease_flags<<<grid_for(cap), kBlock, 0, s>>>(C.xcount, cap, C.xverts, C.xsig, cnt, deg, flag);
        scan_exclusive(flag, cpos, cap, tot + 3, nullptr, tmp, s);
    }
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(DA, buf, s);
        cudaGetLastError();
        return report(ALSUB_ERR_DEVICE, "extraction failed");
    }
    const int Fo = h[0], nnzo = h[1], Vo = h[2], Ko = h[3];
    out.scheme = T.scheme;
    out.V = Vo; out.F = Fo; out.nnz = nnzo; out.K = Ko;
    out.sigma_max = T.mesh->sigma_max;
    out.stream = s;
    if (Fo == 0) {                            // nothing selected: an empty mesh is not a mesh
        dev_free(DA, buf, s);
        return report(ALSUB_ERR_INVALID_ARG, "extraction selected no face");
    }
    e = dev_malloc(DA, &out.d_off, sizeof(int) * (Fo + 1), s);
    if (e == cudaSuccess) e = dev_malloc(DA, &out.d_fv, sizeof(int) * (size_t)nnzo, s);
    if (e == cudaSuccess) e = dev_malloc(DA, &out.d_vmap, sizeof(int) * (size_t)Vo, s);
    if (e == cudaSuccess) e = dev_malloc(DA, &out.d_fmap, sizeof(int) * (size_t)Fo, s);
    if (e == cudaSuccess && Ko) e = dev_malloc(DA, &out.d_cv, sizeof(int) * 2 * (size_t)Ko, s);
    if (e == cudaSuccess && Ko) e = dev_malloc(DA, &out.d_cs, sizeof(float) * (size_t)Ko, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dev_free(DA, buf, s);
        return report(ALSUB_ERR_OOM, "extraction: device allocation failed");
    }
    k_x_fill_faces<<<grid_for(F), kBlock, 0, s>>>(F, off, fv, q, fpos, noff, vpos, out.d_off, out.d_fv, out.d_fmap);
    cudaMemcpyAsync(out.d_off + Fo, tot + 1, sizeof(int), cudaMemcpyDeviceToDevice, s);
    k_x_fill_verts<<<grid_for(V), kBlock, 0, s>>>(V, x, vpos, out.d_vmap);
    if (Ko) k_x_fill_creases<<<grid_for(cap), kBlock, 0, s>>>(cap, flag, cpos, C.xverts, C.xsig, vpos, out.d_cv, out.d_cs);
    dev_free(DA, buf, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
    return ALSUB_OK;
}

void gather_rows(int n, const int *vmap, const float *P, float *out, cudaStream_t s) {
    if (n > 0) k_x_gather<<<grid_for(n), kBlock, 0, s>>>(n, vmap, P, out);
}

}  // namespace alsub
