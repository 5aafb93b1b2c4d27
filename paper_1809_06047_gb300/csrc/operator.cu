// The subdivision operator (Sec. 3.6, "Single SpMV evaluation"): R_l maps the positions of level
// l to those of level l+1, so P_{l+1} = R_l P_l and P_L = R P_0 with R = R_{L-1} ... R_0
// (Eq. singleSpMV). Built on the device in the paper's two stages: count the non-zeros of every
// row, scan, then fill column indices and weights. The weights are the stencils of the eval step
// written out (Catmull-Clark: face row 1/c; edge row 1/4 on the endpoints and 1/(4c) on each face
// vertex (Eq. 2 with Eq. 1 expanded); vertex row (1 - 2/n) p + 1/n^2 sum p_j + 1/n^2 sum f_j
// (Eq. pos_update); Loop and sqrt(3) as in Appendices B and A), with the crease rules as blends.
// Rows are sorted by column and duplicate columns merged, so the composition R_l R can be formed
// row by row with a k-way merge (count, then fill). Transposes (for the adjoint g_l = R_l^T
// g_{l+1}) are built by counting per column and sorting each row, so every matrix is
// deterministic. Apply is a CSR SpMV on packed xyz.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

constexpr int kMaxRow = 192;     // entries of one stencil row before duplicates are merged

struct Csr {
    long long rows = 0, cols = 0, nnz = 0;
    long long *rowptr = nullptr;  // rows + 1
    int *col = nullptr;
    float *w = nullptr;
};

// ---------------------------------------------------------------- stencil rows of one level

struct OpLevel {
    int scheme, l, V, F, E;
    const int *fv, *ce, *tw;       // this level's per-corner arrays (level 0: the Level0 ones)
    Level0 z;
    CreaseList cr;
    bool creases;
    bool bnd;                      // open mesh: twins may be -1, boundary rows come from the list
    int B;                         // boundary list of the level (entries a -> b, successor b -> c)
    const int *bA, *bE, *bS;
};

__device__ __forceinline__ int o_next(const OpLevel &L, int x) {
    if (L.l == 0) return __ldg(L.z.nx + x);
    return L.scheme == ALSUB_CATMULL_CLARK ? quad_next(x) : tri_next(x);
}
__device__ __forceinline__ int o_prev(const OpLevel &L, int x) {
    if (L.l == 0) return __ldg(L.z.pv + x);
    return L.scheme == ALSUB_CATMULL_CLARK ? quad_prev(x) : tri_prev(x);
}
__device__ __forceinline__ int o_twin(const OpLevel &L, int x) { return __ldg(L.tw + x); }
__device__ __forceinline__ int o_edge(const OpLevel &L, int x) { return __ldg(L.ce + x); }
__device__ __forceinline__ int o_vtx(const OpLevel &L, int x) { return __ldg(L.fv + x); }
__device__ __forceinline__ int o_face(const OpLevel &L, int x) {
    if (L.l == 0) return __ldg(L.z.cf + x);
    return L.scheme == ALSUB_CATMULL_CLARK ? (x >> 2) : x / 3;
}
__device__ __forceinline__ void o_face_range(const OpLevel &L, int g, int &s0, int &c) {
    if (L.l == 0) { s0 = __ldg(L.z.off + g); c = __ldg(L.z.off + g + 1) - s0; }
    else if (L.scheme == ALSUB_CATMULL_CLARK) { s0 = 4 * g; c = 4; }
    else { s0 = 3 * g; c = 3; }
}
__device__ __forceinline__ bool o_own(const OpLevel &L, int x) {
    if (L.l == 0) return __ldg(L.z.own + x) != 0;
    if (L.scheme == ALSUB_CATMULL_CLARK) return (x & 3) < 2;
    return loop_own(L.l, x, L.z);
}
__device__ __forceinline__ bool o_vown(const OpLevel &L, int x) {
    if (L.scheme == ALSUB_CATMULL_CLARK) return cc_vown(L.l, x, L.z);
    if (L.scheme == ALSUB_LOOP) return loop_vown(L.l, x, L.z);
    return sqrt3_vown(L.l, x, L.z);
}

struct Row {
    int n;
    bool overflow;
    int c[kMaxRow];
    float w[kMaxRow];
    __device__ void clear() { n = 0; overflow = false; }
    __device__ void add(int col, float wt) {
        if (n < kMaxRow) { c[n] = col; w[n] = wt; n++; }
        else overflow = true;
    }
    __device__ void scale(float s) { for (int i = 0; i < n; i++) w[i] *= s; }
    // sort by column, merge equal columns (in sorted order), drop exact zeros
    __device__ void finish() {
        for (int i = 1; i < n; i++) {
            int ci = c[i]; float wi = w[i]; int k = i - 1;
            while (k >= 0 && c[k] > ci) { c[k + 1] = c[k]; w[k + 1] = w[k]; k--; }
            c[k + 1] = ci; w[k + 1] = wi;
        }
        int m = 0;
        for (int i = 0; i < n;) {
            int ci = c[i]; float s = 0.f;
            while (i < n && c[i] == ci) s += w[i++];
            if (s != 0.f) { c[m] = ci; w[m] = s; m++; }
        }
        n = m;
    }
};

// Valence of the vertex of corner x from its ring walk; 0 when the walk leaves the mesh (a
// boundary vertex), -1 when it does not close within the supported valence.
__device__ int ring_valence(const OpLevel &L, int x) {
    int y = x, n = 0;
    do { n++; y = o_twin(L, o_prev(L, y)); } while (y >= 0 && y != x && n < kMaxValence);
    return y == x ? n : (y < 0 ? 0 : -1);
}

// crease blend of a vertex row: w sharp + (1 - w) smooth for k >= 2 incident creases
__device__ void crease_vertex(const OpLevel &L, int x, Row &R) {
    if (!L.creases) return;
    int y = x, steps = 0, k = 0, n1 = -1, n2 = -1;
    float S = 0.f;
    do {
        const float s = crease_lookup(L.cr, o_edge(L, y));
        if (s > 0.f) {
            const int nb = o_vtx(L, o_next(L, y));
            if (k == 0) n1 = nb; else if (k == 1) n2 = nb;
            k++;
            S += s;
        }
        y = o_twin(L, o_prev(L, y));
        steps++;
    } while (y != x && steps < kMaxValence);
    if (k < 2) return;
    const float sv = S / (float)k;
    const float w = sv < 1.f ? sv : 1.f;
    const int v = o_vtx(L, x);
    R.scale(1.f - w);
    if (k == 2) {
        R.add(n1, 0.125f * w);
        R.add(v, 0.75f * w);
        R.add(n2, 0.125f * w);
    } else {
        R.add(v, w);
    }
}

// crease blend of an edge row: sigma >= 1 midpoint, else (1 - sigma) smooth + sigma midpoint
__device__ void crease_edge(const OpLevel &L, int e, int a, int b, Row &R) {
    if (!L.creases) return;
    const float s = crease_lookup(L.cr, e);
    if (!(s > 0.f)) return;
    const float w = s < 1.f ? s : 1.f;
    R.scale(1.f - w);
    R.add(a, 0.5f * w);
    R.add(b, 0.5f * w);
}

__device__ void face_row(const OpLevel &L, int g, Row &R) {
    int s0, c;
    o_face_range(L, g, s0, c);
    const float wf = 1.f / (float)c;
    for (int k = 0; k < c; k++) R.add(o_vtx(L, s0 + k), wf);
}

// 1: row written; 0: a boundary vertex (its row comes from the boundary list); -1: unsupported.
__device__ int vertex_row(const OpLevel &L, int x, Row &R) {
    const int n = ring_valence(L, x);
    if (n <= 0) return n;
    const int v = o_vtx(L, x);
    const float inv = 1.f / (float)n;
    if (L.scheme == ALSUB_CATMULL_CLARK) {
        const float inv2 = inv * inv;
        R.add(v, 1.f - 2.f * inv);
        int y = x;
        for (int i = 0; i < n; i++) {
            R.add(o_vtx(L, o_next(L, y)), inv2);
            int s0, c;
            o_face_range(L, o_face(L, y), s0, c);
            const float wf = inv2 / (float)c;
            for (int k = 0; k < c; k++) R.add(o_vtx(L, s0 + k), wf);
            y = o_twin(L, o_prev(L, y));
        }
    } else {
        float self, nb;
        if (L.scheme == ALSUB_LOOP) {
            const double t = 0.375 + 0.25 * cos(2.0 * M_PI / n);
            const float beta = (float)((0.625 - t * t) / n);
            self = 1.f - (float)n * beta;
            nb = beta;
        } else {
            const float al = (float)((4.0 - 2.0 * cos(2.0 * M_PI / n)) / 9.0);
            self = 1.f - al;
            nb = al / (float)n;
        }
        R.add(v, self);
        int y = x;
        for (int i = 0; i < n; i++) {
            R.add(o_vtx(L, o_next(L, y)), nb);
            y = o_twin(L, o_prev(L, y));
        }
    }
    if (L.scheme != ALSUB_SQRT3) crease_vertex(L, x, R);
    return 1;
}

__device__ void edge_row(const OpLevel &L, int o, Row &R) {
    const int t = o_twin(L, o);
    const int a = o_vtx(L, o), b = o_vtx(L, t);
    if (L.scheme == ALSUB_CATMULL_CLARK) {
        R.add(a, 0.25f);
        R.add(b, 0.25f);
        const int fs[2] = {o_face(L, o), o_face(L, t)};
        for (int h = 0; h < 2; h++) {
            int s0, c;
            o_face_range(L, fs[h], s0, c);
            const float wf = 0.25f / (float)c;
            for (int k = 0; k < c; k++) R.add(o_vtx(L, s0 + k), wf);
        }
    } else {
        R.add(a, 0.375f);
        R.add(b, 0.375f);
        R.add(o_vtx(L, o_prev(L, o)), 0.125f);
        R.add(o_vtx(L, o_prev(L, t)), 0.125f);
    }
    crease_edge(L, o_edge(L, o), a, b, R);
}

// One thread per face of level l emits the rows this face is responsible for: its face point,
// the edge points of the edges its corners own, the vertex points of the vertices its corners
// are designated for. FILL = false counts, FILL = true writes at rowptr.
template <bool FILL>
__global__ void k_op_rows(OpLevel L, int *cnt, const long long *rowptr, int *col, float *w, int *status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= L.F || failed(status)) return;
    Row R;
    auto emit = [&](int row) {
        R.finish();
        if (R.overflow) { set_status(status, ALSUB_ERR_UNSUPPORTED); return; }
        if (!FILL) { cnt[row] = R.n; return; }
        const long long b = rowptr[row];
        for (int i = 0; i < R.n; i++) { col[b + i] = R.c[i]; w[b + i] = R.w[i]; }
    };
    int s0, c;
    o_face_range(L, r, s0, c);
    const int VF = L.V + L.F;
    if (L.scheme != ALSUB_LOOP) {
        R.clear();
        face_row(L, r, R);
        emit(L.V + r);
    }
    for (int k = 0; k < c; k++) {
        const int x = s0 + k;
        if (L.scheme != ALSUB_SQRT3 && o_own(L, x) && !(L.bnd && o_twin(L, x) < 0)) {
            R.clear();
            edge_row(L, x, R);
            emit((L.scheme == ALSUB_CATMULL_CLARK ? VF : L.V) + o_edge(L, x));
        }
        if (o_vown(L, x)) {
            R.clear();
            const int got = vertex_row(L, x, R);
            if (got < 0 || (got == 0 && !L.bnd)) { set_status(status, ALSUB_ERR_UNSUPPORTED); continue; }
            if (got > 0) emit(o_vtx(L, x));
        }
    }
}

// Boundary rows of a Catmull-Clark or Loop level (Sec. 3.2 "Boundaries"; Loop takes the same
// rules), one thread per boundary-list entry a -> b with successor b -> c: the midpoint row of edge
// (a, b) and the row 3/4 b + 1/8 (a + c) of vertex b (Eq. CC_boundary).
template <bool FILL>
__global__ void k_op_bnd(OpLevel L, int *cnt, const long long *rowptr, int *col, float *w, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.B || failed(status)) return;
    auto clampi = [](int x, int hi) { return min(max(x, 0), hi - 1); };
    const int a = clampi(__ldg(L.bA + i), L.V), e = clampi(__ldg(L.bE + i), L.E);
    const int s1 = clampi(__ldg(L.bS + i), L.B);
    const int b = clampi(__ldg(L.bA + s1), L.V), c = clampi(__ldg(L.bA + clampi(__ldg(L.bS + s1), L.B)), L.V);
    const int re = (L.scheme == ALSUB_CATMULL_CLARK ? L.V + L.F : L.V) + e;
    const int ce[2] = {min(a, b), max(a, b)};
    int cv[3] = {a, b, c};
    float wv[3] = {0.125f, 0.75f, 0.125f};
    for (int p = 1; p < 3; p++)            // sort the vertex row by column
        for (int q = p; q > 0 && cv[q - 1] > cv[q]; q--) {
            int tc = cv[q]; cv[q] = cv[q - 1]; cv[q - 1] = tc;
            float tw = wv[q]; wv[q] = wv[q - 1]; wv[q - 1] = tw;
        }
    if (!FILL) {
        cnt[re] = 2;
        cnt[b] = 3;
        return;
    }
    const long long pe = rowptr[re], pv = rowptr[b];
    for (int k = 0; k < 2; k++) { col[pe + k] = ce[k]; w[pe + k] = 0.5f; }
    for (int k = 0; k < 3; k++) { col[pv + k] = cv[k]; w[pv + k] = wv[k]; }
}

// ---------------------------------------------------------------- transpose

__global__ void k_t_count(long long rows, const long long *__restrict__ rowptr, const int *__restrict__ col,
                          int *cnt) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    for (long long q = rowptr[i]; q < rowptr[i + 1]; q++) atomicAdd(cnt + col[q], 1);
}

__global__ void k_t_fill(long long rows, const long long *__restrict__ rowptr, const int *__restrict__ col,
                         const float *__restrict__ w, const long long *__restrict__ tptr, int *fill,
                         int *tcol, float *tw) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    for (long long q = rowptr[i]; q < rowptr[i + 1]; q++) {
        const int j = col[q];
        const long long p = tptr[j] + atomicAdd(fill + j, 1);
        tcol[p] = (int)i;
        tw[p] = w[q];
    }
}

// atomic fill order is arbitrary: sort each row by column to make the matrix deterministic
__global__ void k_sort_rows(long long rows, const long long *__restrict__ rowptr, int *col, float *w) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const long long b = rowptr[i], n = rowptr[i + 1] - b;
    for (long long a = 1; a < n; a++) {
        const int ca = col[b + a]; const float wa = w[b + a];
        long long k = a - 1;
        while (k >= 0 && col[b + k] > ca) { col[b + k + 1] = col[b + k]; w[b + k + 1] = w[b + k]; k--; }
        col[b + k + 1] = ca; w[b + k + 1] = wa;
    }
}

// ---------------------------------------------------------------- composition C = A B

constexpr int kMaxMerge = kMaxRow;

template <bool FILL>
__global__ void k_gemm(long long rows, const long long *__restrict__ ap, const int *__restrict__ ac,
                       const float *__restrict__ aw, const long long *__restrict__ bp,
                       const int *__restrict__ bc, const float *__restrict__ bw, int *cnt,
                       const long long *__restrict__ cp, int *cc, float *cw, int *status) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const long long a0 = ap[i];
    const int k = (int)(ap[i + 1] - a0);
    if (k > kMaxMerge) { set_status(status, ALSUB_ERR_UNSUPPORTED); return; }
    long long pos[kMaxMerge], end[kMaxMerge];
    for (int h = 0; h < k; h++) {
        const int j = ac[a0 + h];
        pos[h] = bp[j];
        end[h] = bp[j + 1];
    }
    long long out = FILL ? cp[i] : 0;
    int m = 0;
    while (true) {
        int cur = 0x7fffffff;
        for (int h = 0; h < k; h++)
            if (pos[h] < end[h]) cur = min(cur, bc[pos[h]]);
        if (cur == 0x7fffffff) break;
        float s = 0.f;
        for (int h = 0; h < k; h++) {
            if (pos[h] < end[h] && bc[pos[h]] == cur) {
                s += aw[a0 + h] * bw[pos[h]];
                pos[h]++;
            }
        }
        if (FILL) { cc[out + m] = cur; cw[out + m] = s; }
        m++;
    }
    if (!FILL) cnt[i] = m;
}

// ---------------------------------------------------------------- extraction and stacking

// C = X A for an extraction matrix X (row i = e_{vmap[i]}): row i of C is row vmap[i] of A. With
// no A (ap null) A is the identity, and with no map X is too (row i = e_i).
template <bool FILL>
__global__ void k_take_rows(long long rows, const int *__restrict__ vmap, const long long *__restrict__ ap,
                            const int *__restrict__ ac, const float *__restrict__ aw, int *cnt,
                            const long long *__restrict__ cp, int *cc, float *cw) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int j = vmap ? vmap[i] : (int)i;
    if (!ap) {
        if (FILL) { cc[cp[i]] = j; cw[cp[i]] = 1.f; }
        else cnt[i] = 1;
        return;
    }
    const long long a0 = ap[j], n = ap[j + 1] - a0;
    if (!FILL) { cnt[i] = (int)n; return; }
    const long long c0 = cp[i];
    for (long long q = 0; q < n; q++) { cc[c0 + q] = ac[a0 + q]; cw[c0 + q] = aw[a0 + q]; }
}

// rowptr of a block of rows placed at row r0 and entry z0 of a stacked matrix (the last block
// also writes the end)
__global__ void k_rowptr_shift(long long rows, const long long *__restrict__ ap, long long z0, long long *out,
                               bool last) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < rows || (last && i == rows)) out[i] = ap[i] + z0;
}

// ---------------------------------------------------------------- SpMV on packed xyz

// y = A x on xyz rows, S lanes per row: lane k of a row's group takes entries start + k,
// start + k + S, ... (the group reads the row's column ids and weights contiguously), then the
// group sums its partials with shuffles in a fixed order (deterministic). A resident grid walks
// the rows with a grid stride.
template <int S>
__global__ void __launch_bounds__(256) k_spmv(long long rows, const long long *__restrict__ rowptr,
                                              const int *__restrict__ col, const float *__restrict__ w,
                                              const float *__restrict__ x, float *y) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long groups = (long long)gridDim.x * blockDim.x / S;
    const int k = (int)(t % S);
    const long long iters = (rows + groups - 1) / groups;   // the same for every lane (shuffles)
    for (long long n = 0; n < iters; n++) {
        const long long i = t / S + n * groups;
        float3 acc = f3(0.f, 0.f, 0.f);
        if (i < rows)
            for (long long q = rowptr[i] + k, e = rowptr[i + 1]; q < e; q += S)
                acc += __ldg(w + q) * ldp(x, __ldg(col + q));
#pragma unroll
        for (int o = S / 2; o > 0; o >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, S);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, S);
            acc.z += __shfl_down_sync(0xffffffffu, acc.z, o, S);
        }
        if (i < rows && k == 0) stp(y, (int)i, acc);
    }
}

}  // namespace
}  // namespace alsub

using namespace alsub;

struct alsub_operator_s {
    TopoImpl *T = nullptr;
    cudaStream_t stream = nullptr;
    uint32_t flags = 0;
    std::vector<Csr> R, RT;        // per level (ALSUB_OP_CHAIN), and transposes
    Csr C, CT;                     // composite and its transpose (ALSUB_OP_COMPOSE)
    bool has_chain = false, has_comp = false, has_t = false;
    DevAlloc alloc;                // the topology's allocator, copied for the release
    bool matrix_free = false;      // ALSUB_OP_MATRIX_FREE: apply = the stencil kernels on the topology
    float *mf_scratch = nullptr;   // their intermediate levels (the operator's own)
    // applies of a matrix-free operator share its scratch and the topology's launch state: one at a
    // time on the host (mf_lock) and, through mf_done, in order on the device
    std::mutex mf_lock;
    cudaEvent_t mf_done = nullptr;
    // matrix-free transpose (Catmull-Clark, closed meshes): per-vertex coefficients of every level
    // below the last and two intermediate levels of gradients (float4 rows)
    bool mf_t = false;
    std::vector<AdjLevel> adj;
    float *adj_buf = nullptr;
    size_t adj_half = 0;           // floats per intermediate level
    float4 *adj_part = nullptr;    // one per corner of the largest level below the last (any level)
    float *buf = nullptr;          // two intermediate levels of packed xyz for chain applies
    size_t buf_floats = 0;
    int *cnt = nullptr;            // scratch counts
    void *scan_tmp = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;   // with their sizes in bytes
    size_t bytes = 0;
    int sms = 152;                 // SMs of the device (SpMV grid)
    int *status = nullptr;
};

namespace {

template <class T>
alsub_status oalloc(alsub_operator_s &O, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    void *q = nullptr;
    if (dev_malloc(O.alloc, &q, n * sizeof(T), O.stream) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "operator: device allocation failed");
    }
    O.allocs.push_back({q, n * sizeof(T)});
    O.bytes += n * sizeof(T);
    *p = (T *)q;
    return ALSUB_OK;
}

#define OA(ptr, n)                                                \
    do {                                                          \
        alsub_status st_ = oalloc(O, &(ptr), (size_t)(n));        \
        if (st_ != ALSUB_OK) return st_;                          \
    } while (0)

alsub_status read_total(alsub_operator_s &O, long long *dev, long long *host) {
    if (cudaMemcpyAsync(host, dev, sizeof(long long), cudaMemcpyDeviceToHost, O.stream) != cudaSuccess ||
        cudaStreamSynchronize(O.stream) != cudaSuccess) {
        cudaGetLastError();
        return report(ALSUB_ERR_DEVICE, "operator: reading a row count failed");
    }
    return ALSUB_OK;
}

alsub_status check_status(alsub_operator_s &O) {
    int st = 0;
    if (cudaMemcpyAsync(&st, O.status, sizeof(int), cudaMemcpyDeviceToHost, O.stream) != cudaSuccess ||
        cudaStreamSynchronize(O.stream) != cudaSuccess) {
        cudaGetLastError();
        return report(ALSUB_ERR_DEVICE, "operator: synchronisation failed");
    }
    if (st) return report((alsub_status)st, "operator: a row exceeds the supported stencil size");
    return ALSUB_OK;
}

// count -> scan -> allocate -> fill, for any row producer
template <class CountF, class FillF>
alsub_status two_stage(alsub_operator_s &O, Csr &M, long long rows, long long cols, CountF count, FillF fill) {
    M.rows = rows;
    M.cols = cols;
    OA(M.rowptr, rows + 1);
    cudaMemsetAsync(O.cnt, 0, sizeof(int) * (size_t)rows, O.stream);
    count();
    scan_exclusive64(O.cnt, M.rowptr, rows, M.rowptr + rows, O.scan_tmp, O.stream);
    alsub_status st = read_total(O, M.rowptr + rows, &M.nnz);
    if (st) return st;
    st = check_status(O);
    if (st) return st;
    OA(M.col, M.nnz);
    OA(M.w, M.nnz);
    fill();
    return ALSUB_OK;
}

OpLevel op_level(TopoImpl &T, int l) {
    LevelBuf &A = T.L[l];
    OpLevel L;
    L.scheme = T.scheme; L.l = l;
    L.V = (int)A.V; L.F = (int)A.F; L.E = (int)A.E;
    L.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0, T.rn0};
    L.fv = l == 0 ? T.mesh->d_fv : A.fv;
    L.ce = A.ce;
    L.tw = A.tw;
    L.cr = A.cr;
    L.creases = T.scheme != ALSUB_SQRT3 && A.cr.cap > 0;
    L.bnd = T.mesh->B > 0;
    L.B = (int)A.B;
    L.bA = A.bA; L.bE = A.bE; L.bS = A.bS;
    return L;
}

alsub_status build_level(alsub_operator_s &O, int l, Csr &M) {
    TopoImpl &T = *O.T;
    OpLevel L = op_level(T, l);
    const long long rows = T.L[l + 1].V;
    unsigned g = grid_for(L.F);
    cudaStream_t s = O.stream;
    const unsigned gb = grid_for(L.B);
    return two_stage(O, M, rows, T.L[l].V,
        [&] {
            k_op_rows<false><<<g, kBlock, 0, s>>>(L, O.cnt, nullptr, nullptr, nullptr, O.status);
            if (L.B) k_op_bnd<false><<<gb, kBlock, 0, s>>>(L, O.cnt, nullptr, nullptr, nullptr, O.status);
        },
        [&] {
            k_op_rows<true><<<g, kBlock, 0, s>>>(L, O.cnt, M.rowptr, M.col, M.w, O.status);
            if (L.B) k_op_bnd<true><<<gb, kBlock, 0, s>>>(L, O.cnt, M.rowptr, M.col, M.w, O.status);
        });
}

alsub_status build_transpose(alsub_operator_s &O, const Csr &A, Csr &M) {
    cudaStream_t s = O.stream;
    unsigned g = grid_for(A.rows);
    alsub_status st = two_stage(O, M, A.cols, A.rows,
        [&] { k_t_count<<<g, kBlock, 0, s>>>(A.rows, A.rowptr, A.col, O.cnt); },
        [&] {});
    if (st) return st;
    cudaMemsetAsync(O.cnt, 0, sizeof(int) * (size_t)M.rows, s);
    k_t_fill<<<g, kBlock, 0, s>>>(A.rows, A.rowptr, A.col, A.w, M.rowptr, O.cnt, M.col, M.w);
    k_sort_rows<<<grid_for(M.rows), kBlock, 0, s>>>(M.rows, M.rowptr, M.col, M.w);
    return ALSUB_OK;
}

alsub_status build_product(alsub_operator_s &O, const Csr &A, const Csr &B, Csr &M) {
    cudaStream_t s = O.stream;
    unsigned g = grid_for(A.rows);
    return two_stage(O, M, A.rows, B.cols,
        [&] { k_gemm<false><<<g, kBlock, 0, s>>>(A.rows, A.rowptr, A.col, A.w, B.rowptr, B.col, B.w,
                                                O.cnt, nullptr, nullptr, nullptr, O.status); },
        [&] { k_gemm<true><<<g, kBlock, 0, s>>>(A.rows, A.rowptr, A.col, A.w, B.rowptr, B.col, B.w,
                                               O.cnt, M.rowptr, M.col, M.w, O.status); });
}

// M = X A: X the extraction map of `rows` rows (the identity when vmap is null); an A without
// arrays is the identity of A.rows
alsub_status build_take(alsub_operator_s &O, const Csr &A, const int *vmap, long long rows, Csr &M) {
    cudaStream_t s = O.stream;
    unsigned g = grid_for(rows);
    return two_stage(O, M, rows, A.cols,
        [&] { k_take_rows<false><<<g, kBlock, 0, s>>>(rows, vmap, A.rowptr, A.col, A.w, O.cnt,
                                                     nullptr, nullptr, nullptr); },
        [&] { k_take_rows<true><<<g, kBlock, 0, s>>>(rows, vmap, A.rowptr, A.col, A.w, O.cnt,
                                                    M.rowptr, M.col, M.w); });
}

// Lanes per row from the mean row length, about eight entries per lane (measured on the composite
// operator, 16 per row: 2 lanes; the adjoint's transposed levels, ~38 per row: 4 lanes); a
// resident grid of 8 blocks per SM.
#ifndef ALSUB_SPMV_LANES
#define ALSUB_SPMV_LANES 0          // 0: chosen from the mean row length
#endif
void spmv(alsub_operator_s &O, const Csr &M, const float *x, float *y, cudaStream_t s) {
    const double mean = M.rows ? (double)M.nnz / (double)M.rows : 0.0;
    int S = mean > 96 ? 16 : (mean > 48 ? 8 : (mean > 24 ? 4 : (mean > 12 ? 2 : 1)));
    if (ALSUB_SPMV_LANES) S = ALSUB_SPMV_LANES;
    const long long want = (M.rows * S + 255) / 256;
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>(want, 8LL * O.sms));
    if (S == 16) k_spmv<16><<<g, 256, 0, s>>>(M.rows, M.rowptr, M.col, M.w, x, y);
    else if (S == 8) k_spmv<8><<<g, 256, 0, s>>>(M.rows, M.rowptr, M.col, M.w, x, y);
    else if (S == 4) k_spmv<4><<<g, 256, 0, s>>>(M.rows, M.rowptr, M.col, M.w, x, y);
    else if (S == 2) k_spmv<2><<<g, 256, 0, s>>>(M.rows, M.rowptr, M.col, M.w, x, y);
    else k_spmv<1><<<g, 256, 0, s>>>(M.rows, M.rowptr, M.col, M.w, x, y);
    if (O.T) O.T->launches += 1;
}

void free_op(alsub_operator_s *O) {
    if (O->mf_done) {
        cudaEventSynchronize(O->mf_done);
        cudaEventDestroy(O->mf_done);
        O->mf_done = nullptr;
    }
    for (auto &a : O->allocs) dev_free(O->alloc, a.first, O->stream);
    O->allocs.clear();
    O->bytes = 0;
}

// Free the arrays of a matrix that is no longer needed (stream ordered).
void release(alsub_operator_s &O, Csr &M) {
    for (void *p : {(void *)M.rowptr, (void *)M.col, (void *)M.w}) {
        for (size_t i = 0; i < O.allocs.size(); i++) {
            if (O.allocs[i].first != p) continue;
            dev_free(O.alloc, p, O.stream);
            O.bytes -= O.allocs[i].second;
            O.allocs.erase(O.allocs.begin() + i);
            break;
        }
    }
    M = Csr();
}

}  // namespace

extern "C" {

alsub_status alsub_build_operator(alsub_topology_t topo, uint32_t flags, void *stream, alsub_operator_t *out) {
    if (!topo || !out) return report(ALSUB_ERR_INVALID_ARG, "bad operator arguments");
    *out = nullptr;
    if (!(flags & (ALSUB_OP_CHAIN | ALSUB_OP_COMPOSE | ALSUB_OP_MATRIX_FREE)))
        return report(ALSUB_ERR_INVALID_ARG,
                      "flags must ask for ALSUB_OP_CHAIN, ALSUB_OP_COMPOSE and/or ALSUB_OP_MATRIX_FREE");
    TopoImpl &T = *topology_impl(topo);
    if (!T.built) return report(ALSUB_ERR_INVALID_ARG, "topology not built");
    cudaStream_t s = (cudaStream_t)stream;
    const bool want_t = flags & ALSUB_OP_TRANSPOSE;
    // the CSR matrices: per level when a chain, a composite or (for a matrix-free operator) the
    // transposes are asked for
    const bool need_rows = (flags & (ALSUB_OP_CHAIN | ALSUB_OP_COMPOSE)) || want_t;
    if (T.s3f && need_rows)
        return report(ALSUB_ERR_UNSUPPORTED, "operator: the rows of sqrt(3) meshes with boundaries or infinitely "
                                             "sharp creases are evaluated matrix-free only");
    alsub_status st = need_rows ? ensure_helpers(T, s) : ALSUB_OK;
    if (st) return st;
    alsub_operator_s *O = new (std::nothrow) alsub_operator_s();
    if (!O) return report(ALSUB_ERR_OOM, "host allocation failed");
    O->T = &T;
    O->alloc = T.alloc;
    O->stream = s;
    O->flags = flags;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&O->sms, cudaDevAttrMultiProcessorCount, dev);
    }
    auto bail = [&](alsub_status e) { cudaStreamSynchronize(s); free_op(O); delete O; return e; };
    long long vmax = 1;
    for (int l = 0; l <= T.levels; l++) vmax = std::max(vmax, T.L[l].V);
    if (need_rows) {
        if ((st = oalloc(*O, &O->cnt, (size_t)vmax))) return bail(st);
        if ((st = oalloc(*O, (char **)&O->scan_tmp, scan_tmp_bytes(vmax)))) return bail(st);
        if ((st = oalloc(*O, &O->status, 1))) return bail(st);
        cudaMemsetAsync(O->status, 0, sizeof(int), s);
    }
    if (flags & ALSUB_OP_MATRIX_FREE) {
        // the operator applied matrix-free: its rows are the stencils the eval kernels evaluate
        // from the cached topology, so nothing but their scratch is stored
        O->matrix_free = true;
        if (T.scratch_bytes && (st = oalloc(*O, (char **)&O->mf_scratch, T.scratch_bytes))) return bail(st);
        if (cudaEventCreateWithFlags(&O->mf_done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(report(ALSUB_ERR_DEVICE, "operator: event creation failed"));
        }
        if (!want_t && adjoint_supported(T)) {
            // the transpose as a gather per coarse vertex: the levels' edge ids and twins, and
            // each level's per-vertex coefficients (topology only, computed here once)
            if ((st = ensure_helpers(T, s))) return bail(st);
            O->adj.assign(T.levels, AdjLevel());
            long long vmid = 1;
            for (int l = 0; l < T.levels; l++) {
                AdjLevel &P = O->adj[l];
                if ((st = oalloc(*O, (char **)&P.coef, sizeof(float4) * (size_t)T.L[l].V))) return bail(st);
                if ((st = oalloc(*O, &P.corner, (size_t)T.L[l].V))) return bail(st);
                if (l >= 1 && (st = oalloc(*O, &P.pidx, (size_t)T.L[l].nnz))) return bail(st);
                if (adjoint_level_creased(T, l) && (st = oalloc(*O, &P.sh, (size_t)T.L[l].E))) return bail(st);
                adjoint_prepare(T, l, P, s);
                if (l >= 1) vmid = std::max(vmid, T.L[l].V);
            }
            O->adj_half = 4 * (size_t)vmid;
            if ((st = oalloc(*O, &O->adj_buf, 2 * O->adj_half))) return bail(st);
            long long nmax = 1;
            for (int l = 0; l < T.levels; l++)
                nmax = std::max(nmax, l == 0 ? T.L[0].nnz : 4 * T.L[l].V + T.L[l].nnz);
            if ((st = oalloc(*O, (char **)&O->adj_part, sizeof(float4) * (size_t)nmax))) return bail(st);
            O->mf_t = true;
        }
    }
    std::vector<Csr> R(need_rows ? T.levels : 0);
    for (int l = 0; l < (int)R.size(); l++)
        if ((st = build_level(*O, l, R[l]))) return bail(st);
    if ((flags & ALSUB_OP_CHAIN) || (want_t && !(flags & ALSUB_OP_COMPOSE) && O->matrix_free)) {
        O->R = R;
        O->has_chain = true;
        long long vmid = 1;
        for (int l = 1; l < T.levels; l++) vmid = std::max(vmid, T.L[l].V);
        O->buf_floats = 3 * (size_t)vmid;
        if ((st = oalloc(*O, &O->buf, 2 * O->buf_floats))) return bail(st);
        if (want_t) {
            O->RT.resize(T.levels);
            for (int l = 0; l < T.levels; l++)
                if ((st = build_transpose(*O, R[l], O->RT[l]))) return bail(st);
            O->has_t = true;
        }
        if (!(flags & ALSUB_OP_CHAIN)) {        // matrix-free forward: keep the transposes only
            for (Csr &M : O->R) release(*O, M);
            O->R.clear();
            O->has_chain = false;
        }
    }
    if (flags & ALSUB_OP_COMPOSE) {
        if (T.levels == 0) return bail(report(ALSUB_ERR_INVALID_ARG, "no levels to compose"));
        // with no chain kept, each factor and partial product is freed once it has been used
        const bool keep = flags & ALSUB_OP_CHAIN;
        Csr acc = R[0];
        for (int l = 1; l < T.levels; l++) {
            Csr next;
            if ((st = build_product(*O, R[l], acc, next))) return bail(st);
            if (!keep) { release(*O, acc); release(*O, R[l]); }
            acc = next;
        }
        O->C = acc;
        O->has_comp = true;
        if (want_t) {
            if ((st = build_transpose(*O, O->C, O->CT))) return bail(st);
            O->has_t = true;
        }
    }
    if (need_rows && (st = check_status(*O))) return bail(st);
    if (!need_rows && cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return bail(report(ALSUB_ERR_DEVICE, "operator: build failed"));
    }
    if (O->mf_t) {
        // the coefficient kernels check every ring (closed, valence) into the topology's status
        int dst = 0;
        if (cudaMemcpyAsync(&dst, T.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return bail(report(ALSUB_ERR_DEVICE, "operator: build failed"));
        }
        if (dst) return bail(report((alsub_status)dst, "operator: the topology reports an error"));
    }
    *out = O;
    return ALSUB_OK;
}

alsub_status alsub_build_adaptive_operator(const alsub_topology_t *topos, int32_t n, uint32_t flags,
                                           void *stream, alsub_operator_t *out) {
    if (!topos || !out || n < 1) return report(ALSUB_ERR_INVALID_ARG, "bad adaptive operator arguments");
    *out = nullptr;
    if (flags & ~(uint32_t)(ALSUB_OP_TRANSPOSE | ALSUB_OP_STACKED))
        return report(ALSUB_ERR_INVALID_ARG,
                      "adaptive operator: flags may only be ALSUB_OP_TRANSPOSE and ALSUB_OP_STACKED");
    long long vmax = 1;
    for (int k = 0; k < n; k++) {
        if (!topos[k]) return report(ALSUB_ERR_INVALID_ARG, "adaptive operator: NULL topology");
        TopoImpl &T = *topology_impl(topos[k]);
        if (!T.built) return report(ALSUB_ERR_INVALID_ARG, "adaptive operator: topology not built");
        if (T.s3f)
            return report(ALSUB_ERR_UNSUPPORTED, "operator: the rows of sqrt(3) meshes with boundaries or "
                                                 "infinitely sharp creases are evaluated matrix-free only");
        if (k > 0) {
            const TopoImpl &P = *topology_impl(topos[k - 1]);
            if (T.mesh->src_topo != (const void *)&P || T.mesh->src_level != P.levels)
                return report(ALSUB_ERR_INVALID_ARG, "adaptive operator: a round's mesh was not extracted from "
                                                     "the last level of the round before");
        }
        for (int l = 0; l <= T.levels; l++) vmax = std::max(vmax, T.L[l].V);
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < n; k++) {
        TopoImpl &T = *topology_impl(topos[k]);
        // the topology's build and checks (latched on the device) are done before its rows are read
        int tst = 0;
        if (cudaStreamSynchronize(T.stream) != cudaSuccess ||
            cudaMemcpy(&tst, T.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return report(ALSUB_ERR_DEVICE, "adaptive operator: reading a topology's status failed");
        }
        if (tst) return report((alsub_status)tst, "adaptive operator: a topology reports an error");
        if (T.levels > 0) {
            alsub_status st = ensure_helpers(T, s);
            if (st) return st;
        }
    }
    alsub_operator_s *O = new (std::nothrow) alsub_operator_s();
    if (!O) return report(ALSUB_ERR_OOM, "host allocation failed");
    O->alloc = topology_impl(topos[0])->alloc;
    O->stream = s;
    O->flags = flags;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&O->sms, cudaDevAttrMultiProcessorCount, dev);
    }
    auto bail = [&](alsub_status e) { cudaStreamSynchronize(s); free_op(O); delete O; return e; };
    alsub_status st;
    if ((st = oalloc(*O, &O->cnt, (size_t)vmax))) return bail(st);
    if ((st = oalloc(*O, (char **)&O->scan_tmp, scan_tmp_bytes(vmax)))) return bail(st);
    if ((st = oalloc(*O, &O->status, 1))) return bail(st);
    cudaMemsetAsync(O->status, 0, sizeof(int), s);
    const bool stacked = flags & ALSUB_OP_STACKED;
    // C: the rows so far over the control points (no arrays: the identity); parts: each round's
    // rows when stacked (kept, so C is not released once it is one)
    Csr C;
    C.rows = C.cols = topology_impl(topos[0])->L[0].V;
    bool c_kept = false;
    std::vector<Csr> parts;
    auto replace = [&](Csr next) {
        if (!c_kept) release(*O, C);
        C = next;
        c_kept = false;
    };
    for (int k = 0; k < n; k++) {
        TopoImpl &T = *topology_impl(topos[k]);
        O->T = &T;
        if (k > 0) {                            // X^(k): the rows of the kept vertices
            Csr X;
            if ((st = build_take(*O, C, T.mesh->d_vmap, T.L[0].V, X))) return bail(st);
            replace(X);
        }
        for (int l = 0; l < T.levels; l++) {    // R^(k), level by level
            Csr Rl;
            if ((st = build_level(*O, l, Rl))) return bail(st);
            if (!C.rowptr) {
                C = Rl;                         // the identity times R_l
                continue;
            }
            Csr next;
            if ((st = build_product(*O, Rl, C, next))) return bail(st);
            release(*O, Rl);
            replace(next);
        }
        if (stacked) {
            if (!C.rowptr) {                    // a round of no levels on the control mesh
                Csr I;
                if ((st = build_take(*O, C, nullptr, C.rows, I))) return bail(st);
                C = I;
            }
            parts.push_back(C);
            c_kept = true;
        }
    }
    O->T = nullptr;                             // the operator keeps nothing of the topologies
    if (stacked) {
        Csr S;
        S.cols = C.cols;
        for (const Csr &p : parts) { S.rows += p.rows; S.nnz += p.nnz; }
        if ((st = oalloc(*O, &S.rowptr, S.rows + 1)) || (st = oalloc(*O, &S.col, S.nnz)) ||
            (st = oalloc(*O, &S.w, S.nnz)))
            return bail(st);
        long long r0 = 0, z0 = 0;
        for (size_t i = 0; i < parts.size(); i++) {
            const Csr &p = parts[i];
            const bool last = i + 1 == parts.size();
            k_rowptr_shift<<<grid_for(p.rows + 1), kBlock, 0, s>>>(p.rows, p.rowptr, z0, S.rowptr + r0, last);
            cudaMemcpyAsync(S.col + z0, p.col, sizeof(int) * (size_t)p.nnz, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(S.w + z0, p.w, sizeof(float) * (size_t)p.nnz, cudaMemcpyDeviceToDevice, s);
            r0 += p.rows;
            z0 += p.nnz;
        }
        for (Csr &p : parts) release(*O, p);
        C = S;
    } else if (!C.rowptr) {                     // one round of no levels: R is the identity
        Csr I;
        if ((st = build_take(*O, C, nullptr, C.rows, I))) return bail(st);
        C = I;
    }
    O->C = C;
    O->has_comp = true;
    if (flags & ALSUB_OP_TRANSPOSE) {
        if ((st = build_transpose(*O, O->C, O->CT))) return bail(st);
        O->has_t = true;
    }
    if ((st = check_status(*O))) return bail(st);
    *out = O;
    return ALSUB_OK;
}

alsub_status alsub_operator_info(alsub_operator_t op, int32_t level, int64_t *rows, int64_t *cols,
                                 int64_t *nnz, const int64_t **rowptr_dev, const int32_t **col_dev,
                                 const float **w_dev) {
    if (!op) return report(ALSUB_ERR_INVALID_ARG, "NULL operator");
    const Csr *M = nullptr;
    if (level < 0) { if (op->has_comp) M = &op->C; }
    else if (op->has_chain && level < (int)op->R.size()) M = &op->R[level];
    if (!M) return report(ALSUB_ERR_INVALID_ARG, "the operator holds no such matrix");
    if (rows) *rows = M->rows;
    if (cols) *cols = M->cols;
    if (nnz) *nnz = M->nnz;
    if (rowptr_dev) *rowptr_dev = (const int64_t *)M->rowptr;
    if (col_dev) *col_dev = M->col;
    if (w_dev) *w_dev = M->w;
    return ALSUB_OK;
}

alsub_status alsub_apply_operator(alsub_operator_t op, const float *P0, float *PL, void *stream) {
    if (!op || !P0 || !PL) return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (op->matrix_free) {
        std::lock_guard<std::mutex> g(op->mf_lock);
        cudaStreamWaitEvent(s, op->mf_done, 0);        // the previous apply's scratch use is done
        alsub_status st = refine_call(*op->T, P0, PL, op->mf_scratch, s);
        cudaEventRecord(op->mf_done, s);
        return st;
    }
    if (op->has_comp) {
        spmv(*op, op->C, P0, PL, s);
    } else {
        const int L = (int)op->R.size();
        const float *in = P0;
        for (int l = 0; l < L; l++) {
            float *o = l == L - 1 ? PL : op->buf + op->buf_floats * (l & 1);
            spmv(*op, op->R[l], in, o, s);
            in = o;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
}

alsub_status alsub_apply_operator_transpose(alsub_operator_t op, const float *gL, float *g0, void *stream) {
    if (!op || !gL || !g0) return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (!op->has_t && op->mf_t) {
        // g_l = R_l^T g_{l+1} gathered per coarse vertex, level by level from the last
        std::lock_guard<std::mutex> g(op->mf_lock);
        cudaStreamWaitEvent(s, op->mf_done, 0);        // the previous apply's buffers are free
        TopoImpl &T = *op->T;
        const int L = T.levels;
        for (int l = L - 1; l >= 0; l--) {
            const float *G = l == L - 1 ? gL : op->adj_buf + op->adj_half * ((l + 1) & 1);
            float *gl = l == 0 ? g0 : op->adj_buf + op->adj_half * (l & 1);
            adjoint_step(T, l, G, l + 1 < L, gl, l > 0, op->adj[l], op->adj_part, s);
        }
        cudaEventRecord(op->mf_done, s);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
    }
    if (!op->has_t) return report(ALSUB_ERR_INVALID_ARG, "operator built without ALSUB_OP_TRANSPOSE");
    if (op->has_comp) {
        spmv(*op, op->CT, gL, g0, s);
    } else {
        const int L = (int)op->RT.size();
        const float *in = gL;
        for (int l = L - 1, i = 0; l >= 0; l--, i++) {
            float *o = l == 0 ? g0 : op->buf + op->buf_floats * (i & 1);
            spmv(*op, op->RT[l], in, o, s);
            in = o;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
}

alsub_status alsub_operator_bytes(alsub_operator_t op, size_t *bytes) {
    if (!op || !bytes) return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    *bytes = op->bytes;
    return ALSUB_OK;
}

alsub_status alsub_operator_destroy(alsub_operator_t op) {
    if (!op) return ALSUB_OK;
    free_op(op);
    delete op;
    return ALSUB_OK;
}

}  // extern "C"
