// Regular-patch evaluation (Sec. 3.4, feature-adaptive subdivision): a Catmull-Clark face whose
// 3 x 3 block of faces is regular (9 quads around 4 interior vertices of valence 4, no live crease
// at its 16 vertices) is a bicubic B-spline patch over its 4 x 4 control net, whose limit surface
// is evaluated directly instead of being subdivided further.
//
// Control net: the face [v0, v1, v2, v3] spans grid cells (1..2, 1..2), u along v0 -> v1, v along
// v0 -> v3. Around each corner vertex v_k the ring walk x <- twin(prev(x)) visits its four faces;
// each, started at v_k, gives three of the vertices around v_k at fixed offsets in the corner's own
// (u, v) frame, so the four walks place all 16 points (the edge-adjacent ones twice, consistently).
// Evaluation: S(u, v) = sum_ij B_i(u) B_j(v) P_ij with the uniform cubic B-spline basis
// B_0 = (1-t)^3 / 6, B_1 = (3t^3 - 6t^2 + 4) / 6, B_2 = (-3t^3 + 3t^2 + 3t + 1) / 6, B_3 = t^3 / 6.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

// corner access of one level: level 0 (general faces) or a quad level with stored twins
struct PatchAcc {
    int l;
    const int *off, *fv, *nx, *pv, *cf, *tw;  // level 0 uses off / nx / pv / cf; levels >= 1 quads
    __device__ int next(int x) const { return l == 0 ? __ldg(nx + x) : quad_next(x); }
    __device__ int prev(int x) const { return l == 0 ? __ldg(pv + x) : quad_prev(x); }
    __device__ int vtx(int x) const { return __ldg(fv + x); }
    __device__ int twin(int x) const { return __ldg(tw + x); }
    __device__ bool quad_at(int x) const {          // the face of corner x is a quad
        if (l > 0) return true;
        const int g = __ldg(cf + x);
        return __ldg(off + g + 1) - __ldg(off + g) == 4;
    }
    __device__ int first(int r, int &order) const {
        if (l > 0) { order = 4; return 4 * r; }
        const int s = __ldg(off + r);
        order = __ldg(off + r + 1) - s;
        return s;
    }
};

// The 16 control vertices of face r (grid[4 j + i] for grid cell (i, j)), or false when the face
// is not regular.
__device__ bool control_net(const PatchAcc &A, int r, const unsigned char *__restrict__ crease_v, int *grid) {
    int order;
    const int c0 = A.first(r, order);
    if (order != 4) return false;
    // corner k: base cell and the (u, v) axes of its frame in grid units
    const int bx[4] = {1, 2, 2, 1}, by[4] = {1, 1, 2, 2};
    const int ux[4] = {1, 0, -1, 0}, uy[4] = {0, 1, 0, -1};
    const int vx[4] = {0, -1, 0, 1}, vy[4] = {1, 0, -1, 0};
    // offsets (a, b) in the corner frame of the vertices the ring faces 1, 2, 3 contribute
    // (face s started at the corner vertex is [v, a_s, b_s, c_s]): b1 (-1, 1), c1 (-1, 0),
    // b2 (-1, -1), c2 (0, -1), b3 (1, -1)
    int x = c0;
    for (int k = 0; k < 4; k++, x = A.next(x)) {
        const int v = A.vtx(x);
        int y = x, steps = 0;
        int ring[4];
        do {
            if (!A.quad_at(y)) return false;
            if (steps < 4) ring[steps] = y;
            const int t = A.twin(A.prev(y));
            if (t < 0) return false;                 // a boundary vertex
            y = t;
            steps++;
        } while (y != x && steps <= 4);
        if (y != x || steps != 4) return false;      // valence 4
        auto put = [&](int a, int b, int vert) {
            const int gx = bx[k] + a * ux[k] + b * vx[k], gy = by[k] + a * uy[k] + b * vy[k];
            grid[4 * gy + gx] = vert;
        };
        put(0, 0, v);
        const int f1 = ring[1], f2 = ring[2], f3 = ring[3];
        put(-1, 1, A.vtx(A.next(A.next(f1))));
        put(-1, 0, A.vtx(A.prev(f1)));
        put(-1, -1, A.vtx(A.next(A.next(f2))));
        put(0, -1, A.vtx(A.prev(f2)));
        put(1, -1, A.vtx(A.next(A.next(f3))));
    }
    if (crease_v)
        for (int q = 0; q < 16; q++)
            if (crease_v[grid[q]]) return false;
    return true;
}

__global__ void k_patch_flags(PatchAcc A, int F, const unsigned char *__restrict__ crease_v, unsigned char *flags,
                              unsigned long long *count) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= F) return;
    int grid[16];
    const bool ok = control_net(A, r, crease_v, grid);
    flags[r] = ok ? 1 : 0;
    if (ok) atomicAdd(count, 1ull);
}

__global__ void k_patch_nets(PatchAcc A, int n, const int *__restrict__ faces, int F,
                             const unsigned char *__restrict__ crease_v, int *nets) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = faces[i];
    int grid[16];
    const bool ok = r >= 0 && r < F && control_net(A, r, crease_v, grid);
    for (int q = 0; q < 16; q++) nets[16 * (size_t)i + q] = ok ? grid[q] : -1;
}

__device__ __forceinline__ void cubic_basis(float t, float *B) {
    const float s = 1.f - t, t2 = t * t, t3 = t2 * t;
    B[0] = s * s * s * (1.f / 6.f);
    B[1] = (3.f * t3 - 6.f * t2 + 4.f) * (1.f / 6.f);
    B[2] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * (1.f / 6.f);
    B[3] = t3 * (1.f / 6.f);
}

// one thread per sample (patch i, row b, column a)
__global__ void k_patch_eval(long long total, int samples, const int *__restrict__ nets, const float *__restrict__ P,
                             float *out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int per = samples * samples;
    const long long i = t / per;
    const int rem = (int)(t - i * per), b = rem / samples, a = rem - b * samples;
    const int *net = nets + 16 * i;
    float3 acc = f3(0.f, 0.f, 0.f);
    if (__ldg(net) < 0) {
        acc = f3(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    } else {
        const float inv = samples > 1 ? 1.f / (float)(samples - 1) : 0.f;
        float Bu[4], Bv[4];
        cubic_basis((float)a * inv, Bu);
        cubic_basis((float)b * inv, Bv);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float3 row = f3(0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 4; q++) row += Bu[q] * ldp(P, __ldg(net + 4 * j + q));
            acc += Bv[j] * row;
        }
    }
    out[3 * t + 0] = acc.x;
    out[3 * t + 1] = acc.y;
    out[3 * t + 2] = acc.z;
}

// A block per patch for samples^2 <= 1024 (tpp threads; the kernel takes several patches per block,
// kPatchSlots at most): the 16 control points into shared memory, then its 4 rows interpolated along u
// (R_j(a) = sum_i B_i(u_a) P_ij), then each sample S(a, b) = sum_j B_j(v_b) R_j(a); a patch's
// samples are written as one contiguous run.
constexpr int kPatchSlots = 1;
__global__ void __launch_bounds__(1024) k_patch_eval_block(int n, int samples, int tpp, const int *__restrict__ nets,
                                                           const float *__restrict__ P, float *out) {
    __shared__ float4 sp[kPatchSlots][16];
    __shared__ float4 sr[kPatchSlots][4][32];
    const int slot = threadIdx.x / tpp, lt = threadIdx.x - slot * tpp;
    const long long i = (long long)blockIdx.x * (blockDim.x / tpp) + slot;
    const int per = samples * samples;
    const float inv = samples > 1 ? 1.f / (float)(samples - 1) : 0.f;
    const bool live = i < n;
    if (live && lt < 16) {
        const int id = __ldg(nets + 16 * i + lt);
        const float nan = __int_as_float(0x7fc00000);
        const float3 q = id < 0 ? f3(nan, nan, nan) : ldp(P, id);
        sp[slot][lt] = make_float4(q.x, q.y, q.z, 0.f);
    }
    __syncthreads();
    if (live && lt < 4 * samples) {
        const int j = lt / samples, a = lt - j * samples;
        float B[4];
        cubic_basis((float)a * inv, B);
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float4 c = sp[slot][4 * j + q];
            r.x += B[q] * c.x; r.y += B[q] * c.y; r.z += B[q] * c.z;
        }
        sr[slot][j][a] = r;
    }
    __syncthreads();
    if (!live || lt >= per) return;
    const int b = lt / samples, a = lt - b * samples;
    float B[4];
    cubic_basis((float)b * inv, B);
    float3 acc = f3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float4 r = sr[slot][j][a];
        acc += B[j] * f3(r.x, r.y, r.z);
    }
    float *o = out + 3 * ((size_t)i * per + lt);
    o[0] = acc.x;
    o[1] = acc.y;
    o[2] = acc.z;
}

__global__ void k_patch_crease_flags(const int *__restrict__ count, int cap, const int *__restrict__ cv,
                                     const float *__restrict__ cs, unsigned char *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap || i >= *count || !(cs[i] > 0.f)) return;
    flag[cv[2 * i]] = 1;
    flag[cv[2 * i + 1]] = 1;
}

// Corner access of level l and (in *crease_v, a V_l-byte device array from the caller's temporary
// `buf`) the vertices touched by its live creases; false when the level keeps no twins.
bool patch_setup(TopoImpl &T, int l, cudaStream_t s, PatchAcc *A, unsigned char *crease_v) {
    const LevelBuf &L = T.L[l];
    if (!L.tw) return false;
    if (l == 0) *A = PatchAcc{0, T.mesh->d_off, L.fv, T.nx0, T.pv0, T.cf0, L.tw};
    else *A = PatchAcc{l, nullptr, L.fv, nullptr, nullptr, nullptr, L.tw};
    cudaMemsetAsync(crease_v, 0, (size_t)L.V, s);
    const CreaseList &C = L.cr;
    if (C.cap > 0) {
        T.launches += crease_export(T, l, s);
        k_patch_crease_flags<<<grid_for(C.cap), kBlock, 0, s>>>(C.xcount, (int)C.cap, C.xverts, C.xsig, crease_v);
    }
    return true;
}

alsub_status patch_args(alsub_topology_t topo, int32_t level, TopoImpl **Tout, cudaStream_t s) {
    if (!topo) return report(ALSUB_ERR_INVALID_ARG, "NULL topology");
    TopoImpl &T = *topology_impl(topo);
    if (T.scheme != ALSUB_CATMULL_CLARK) return report(ALSUB_ERR_UNSUPPORTED, "bicubic patches are Catmull-Clark's");
    if (!T.built) return report(ALSUB_ERR_INVALID_ARG, "topology not built");
    if (level < 0 || level >= T.levels)
        return report(ALSUB_ERR_INVALID_ARG, "patches need a level below the topology's last (its twins)");
    alsub_status st = ensure_helpers(T, s);
    if (st != ALSUB_OK) return st;
    *Tout = &T;
    return ALSUB_OK;
}

}  // namespace

}  // namespace alsub

using namespace alsub;

extern "C" {

alsub_status alsub_topology_regular_faces(alsub_topology_t topo, int32_t level, uint8_t *flags_dev, int64_t *count,
                                          void *stream) {
    if (!flags_dev) return report(ALSUB_ERR_INVALID_ARG, "NULL flags");
    cudaStream_t s = (cudaStream_t)stream;
    TopoImpl *T = nullptr;
    alsub_status st = patch_args(topo, level, &T, s);
    if (st != ALSUB_OK) return st;
    const LevelBuf &L = T->L[level];
    char *buf = nullptr;
    if (dev_malloc(T->alloc, &buf, (size_t)L.V + 64, s) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "patches: device allocation failed");
    }
    unsigned long long *cnt = (unsigned long long *)buf;
    unsigned char *crease_v = (unsigned char *)buf + 64;
    PatchAcc A;
    if (!patch_setup(*T, level, s, &A, crease_v)) {
        dev_free(T->alloc, buf, s);
        return report(ALSUB_ERR_INVALID_ARG, "the level keeps no twins");
    }
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    k_patch_flags<<<grid_for(L.F), kBlock, 0, s>>>(A, (int)L.F, crease_v, flags_dev, cnt);
    T->launches += 1;
    unsigned long long h = 0;
    cudaError_t e = cudaSuccess;
    if (count) {
        e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *count = (int64_t)h;
    }
    dev_free(T->alloc, buf, s);
    if (e != cudaSuccess) return report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
    e = cudaGetLastError();
    return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
}

alsub_status alsub_topology_eval_patches(alsub_topology_t topo, int32_t level, int32_t n, const int32_t *faces_dev,
                                         const float *P_dev, int32_t samples, float *out_dev, void *stream) {
    if (n < 0 || samples < 1 || samples > 1024 || (n > 0 && (!faces_dev || !P_dev || !out_dev)))
        return report(ALSUB_ERR_INVALID_ARG, "bad patch arguments");
    cudaStream_t s = (cudaStream_t)stream;
    TopoImpl *T = nullptr;
    alsub_status st = patch_args(topo, level, &T, s);
    if (st != ALSUB_OK || n == 0) return st;
    const LevelBuf &L = T->L[level];
    char *buf = nullptr;
    const size_t net_bytes = 64 * (size_t)n;
    if (dev_malloc(T->alloc, &buf, net_bytes + (size_t)L.V + 16, s) != cudaSuccess) {
        return report(ALSUB_ERR_OOM, "patches: device allocation failed");
    }
    int *nets = (int *)buf;
    unsigned char *crease_v = (unsigned char *)buf + net_bytes;
    PatchAcc A;
    if (!patch_setup(*T, level, s, &A, crease_v)) {
        dev_free(T->alloc, buf, s);
        return report(ALSUB_ERR_INVALID_ARG, "the level keeps no twins");
    }
    k_patch_nets<<<grid_for(n), kBlock, 0, s>>>(A, n, faces_dev, (int)L.F, crease_v, nets);
    const long long total = (long long)n * samples * samples;
    if (samples <= 32) {
        const int tpp = std::max(64, ((samples * samples + 31) / 32) * 32);
        // one patch per block measured faster than four (1024 threads, 2 resident blocks per SM)
        const int per_block = 1;
        k_patch_eval_block<<<(n + per_block - 1) / per_block, per_block * tpp, 0, s>>>(n, samples, tpp, nets, P_dev,
                                                                                      out_dev);
    } else {
        k_patch_eval<<<(unsigned)((total + kBlock - 1) / kBlock), kBlock, 0, s>>>(total, samples, nets, P_dev, out_dev);
    }
    T->launches += 2;
    dev_free(T->alloc, buf, s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
}

}  // extern "C"
