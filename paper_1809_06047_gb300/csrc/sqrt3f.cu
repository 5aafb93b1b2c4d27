// sqrt(3) refinement with feature edges: boundaries and infinitely sharp creases (Appendix A gives
// neither; the treatment follows Kobbelt 2000, Sec. 4). The closed-mesh kernels of tri.cu derive
// every index from closed-form rules that assume every edge flips; a feature edge never flips, so
// meshes with features take this general path, one step at a time with the arrays of every level
// below the last stored:
//   fv  triangle rows (3 ints); tw  per-corner twin (a boundary corner holds -1 - its rank among the
//   level's boundary corners in corner order); fm  per-triangle byte, bit j set when corner j's
//   edge is a feature edge; vc  per vertex, one of its outgoing corners (the level-0 designated
//   corner, then carried to the child that keeps the vertex, so no search is needed); and the
//   level's crease edges as a list (appended by the step that makes the level).
// Steps alternate, by the level they start from:
//   first step of a pair (even level l): a face point at |v| + i for every triangle i; corner k of
//     (k, l, m) gives (p_k, f_{F(l,k)}, f_i), or (p_k, p_l, f_i) when k -> l is a feature edge;
//   second step (odd level l): a triangle with a feature edge a -> b (one at most, by construction)
//     gets no face point; the edge splits into three at q1 (near a, in the triangle's slot |v| + i)
//     and q2 (near b: the slot of the triangle across a crease, or |v| + |f| + rank for a boundary
//     edge), and the triangle into (a, q1, c), (q1, q2, c), (q2, b, c); an edge flips only between
//     two triangles with face points.
// Positions: face points are barycenters; curve vertices (two feature edges) stay on the first step
// and take (4, 19, 4) / 27 on the second, corners (three or more) stay, every other vertex takes Eq.
// sqrt2; q1, q2 take the ternary cubic B-spline masks (1, 16, 10) / 27 and (10, 16, 1) / 27, the
// neighbour beyond a curve end (a corner or a dart) read as its mirror 2 p_end - p_next.
// Per step: a vertex pass (one thread per vertex: its ring from its corner, its feature neighbours,
// its position) and a triangle pass (one thread per triangle: children, their twins, flags and
// corners, the level's crease list, face points and feature-edge points).
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

// alpha_n of Eq. alpha, (4 - 2 cos(2 pi / n)) / 9, computed on the host in double once
__constant__ float c_s3f_alpha[kMaxValence + 1];

}  // namespace

void s3f_upload_tables() {
    static std::once_flag once;
    std::call_once(once, [] {
        static float al[kMaxValence + 1];
        al[0] = 0.f;
        for (int n = 1; n <= kMaxValence; n++) al[n] = (float)((4.0 - 2.0 * cos(2.0 * M_PI / n)) / 9.0);
        cudaMemcpyToSymbol(c_s3f_alpha, al, sizeof(al));
    });
}

namespace {

struct S3Args {
    int l, V, F;
    bool odd;                        // first step of a pair (from an even level)
    const int *fv, *tw, *vc;         // level l
    const unsigned char *fm;
    int4 *vi;                        // per vertex of level l: feature valency, feature neighbours
    const float *P;
    float *Pn;
    bool in4, out4;
    int *fvn, *twn, *vcn;            // level l + 1 (twn, fmn, vcn null when it is the last level)
    unsigned char *fmn;
    int *ccount, *cverts;            // level l + 1's crease list
    float *csig;
    int ccap;
    int *status;
    // level l - 1 (l >= 1): the step that made level l, and whether it was a first step
    const int *pfv = nullptr, *ptw = nullptr;
    const unsigned char *pfm = nullptr;
    int Vp = 0, Fp = 0;
    bool podd = false;
    // level l - 2 (l >= 2): twins and feature bits, and whether the step from it was a first step
    const int *p2tw = nullptr;
    const unsigned char *p2fm = nullptr;
    int V2 = 0, F2 = 0;
    bool p2odd = false;
};

__device__ __forceinline__ int t_next(int x) { const int q = x / 3; return 3 * q + (x - 3 * q == 2 ? 0 : x - 3 * q + 1); }
__device__ __forceinline__ int t_prev(int x) { const int q = x / 3; return 3 * q + (x - 3 * q == 0 ? 2 : x - 3 * q - 1); }
__device__ __forceinline__ bool feat(const unsigned char *fm, int x) {
    const int q = x / 3;
    return (__ldg(fm + q) >> (x - 3 * q)) & 1;
}

// One vertex per thread: its ring from its corner (the open fan of a boundary vertex walked both
// ways), its feature edges, and with EVAL its refined position.
template <bool EVAL>
__global__ void __launch_bounds__(kBlock) k_s3f_vert(S3Args a) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V || failed(a.status)) return;
    if (a.pfv && v >= a.Vp && v < a.Vp + a.Fp) {
        // The face point f_T of triangle T of level l - 1, when all three of T's edges flipped on
        // the step that made it (T and, after a second step, the triangles across have no feature
        // edge; none is a boundary edge): its ring alternates T's vertices and the face points
        // across T's edges, v_0, f_N0, v_1, f_N1, v_2, f_N2 (the order the walk from its corner,
        // child 0's corner 2, takes), none of its edges is a feature edge. Read from level l - 1
        // in two round trips instead of a walk of six twins; the same sum in the same order.
        const int T = v - a.Vp;
        const int mT = __ldg(a.pfm + T) & 7;
        int vt[3], tn[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            vt[j] = __ldg(a.pfv + 3 * T + j);
            tn[j] = __ldg(a.ptw + 3 * T + j);
        }
        bool flat = mT == 0 && tn[0] >= 0 && tn[1] >= 0 && tn[2] >= 0;
        if (flat && !a.podd) {
#pragma unroll
            for (int j = 0; j < 3; j++) flat = flat && (__ldg(a.pfm + tn[j] / 3) & 7) == 0;
        }
        if (flat) {
            a.vi[v] = make_int4(0, -1, -1, 0);
            if (!EVAL) return;
            float3 sum = f3(0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                sum += ldpv(a.P, vt[j], a.in4);
                sum += ldpv(a.P, a.Vp + tn[j] / 3, a.in4);
            }
            const float al = c_s3f_alpha[6];
            stpv(a.Pn, v, (1.0f - al) * ldpv(a.P, v, a.in4) + (al / 6.0f) * sum, a.out4);
            return;
        }
    }
    if (a.p2tw && v >= a.V2 && v < a.V2 + a.F2) {
        // The face point f_T of triangle T of level l - 2, when T's edges all flipped on the step
        // that made it and the six edges at f_T flipped on the next: its ring on level l is the
        // face points of its six triangles on level l - 1, the children 3T + j of T's corners and
        // t_j of the corners across (t_j = T's twins), in the walk's order from its corner: f(t_2),
        // f(3T), f(t_0), f(3T + 1), f(t_1), f(3T + 2). None of its edges is a feature edge.
        const int T = v - a.V2;
        int tn[3];
#pragma unroll
        for (int j = 0; j < 3; j++) tn[j] = __ldg(a.p2tw + 3 * T + j);
        bool flat = (__ldg(a.p2fm + T) & 7) == 0 && tn[0] >= 0 && tn[1] >= 0 && tn[2] >= 0;
        if (flat) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                // a second step flips an edge only between two triangles with face points
                if (!a.p2odd) flat = flat && (__ldg(a.p2fm + tn[j] / 3) & 7) == 0;
                if (!a.podd) flat = flat && (__ldg(a.pfm + 3 * T + j) & 7) == 0 && (__ldg(a.pfm + tn[j]) & 7) == 0;
            }
        }
        if (flat) {
            a.vi[v] = make_int4(0, -1, -1, 0);
            if (!EVAL) return;
            const int q[6] = {tn[2], 3 * T, tn[0], 3 * T + 1, tn[1], 3 * T + 2};
            float3 sum = f3(0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 6; u++) sum += ldpv(a.P, a.Vp + q[u], a.in4);
            const float al = c_s3f_alpha[6];
            stpv(a.Pn, v, (1.0f - al) * ldpv(a.P, v, a.in4) + (al / 6.0f) * sum, a.out4);
            return;
        }
    }
    const int x = __ldg(a.vc + v);
    int k = 0, n1 = -1, n2 = -1, n = 0;
    float3 sum = f3(0.f, 0.f, 0.f);
    auto neighbour = [&](int w, bool feature) {
        if (EVAL) sum += ldpv(a.P, w, a.in4);
        n++;
        if (feature) {
            if (k == 0) n1 = w;
            else if (k == 1) n2 = w;
            k++;
        }
    };
    // the ring eight corners per round: each corner's neighbour and feature bit are loaded as soon
    // as the chain of twins (the only dependent loads) reaches it, and the round's positions after
    // the chain, so a valence-6 vertex waits for the chain plus about two round trips
    int y = x;
    bool open = false, done = false;
    while (!done && n < kMaxValence) {
        int w[8];
        unsigned char f[8];
        bool use[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            use[q] = !done;
            w[q] = 0;
            f[q] = 0;
            if (!done) {
                w[q] = __ldg(a.fv + t_next(y));
                const int qq = y / 3;
                f[q] = (unsigned char)((__ldg(a.fm + qq) >> (y - 3 * qq)) & 1);
                const int t = __ldg(a.tw + t_prev(y));
                if (t < 0) {
                    open = true;             // y stays the corner whose previous edge is open
                    done = true;
                } else {
                    y = t;
                    done = y == x || n + q + 1 >= kMaxValence;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (use[q]) neighbour(w[q], f[q] != 0);
    }
    if (open) {
        // the fan ends at an incoming boundary edge u -> v; then the corners before x
        neighbour(__ldg(a.fv + t_prev(y)), true);
        y = x;
        while (n < kMaxValence) {
            const int t = __ldg(a.tw + y);
            if (t < 0) break;
            y = t_next(t);
            neighbour(__ldg(a.fv + t_next(y)), feat(a.fm, y));
        }
    }
    if (n >= kMaxValence) {
        set_status(a.status, ALSUB_ERR_UNSUPPORTED);
        return;
    }
    a.vi[v] = make_int4(k, n1, n2, 0);
    if (!EVAL) return;
    const float3 p = ldpv(a.P, v, a.in4);
    float3 q;
    if (k >= 3 || (a.odd && k == 2)) {
        q = p;                                         // a corner; a curve vertex on a first step
    } else if (k == 2) {
        q = (4.0f / 27.0f) * (ldpv(a.P, n1, a.in4) + ldpv(a.P, n2, a.in4)) + (19.0f / 27.0f) * p;
    } else {
        const float al = c_s3f_alpha[n];
        q = (1.0f - al) * p + (al / (float)n) * sum;
    }
    stpv(a.Pn, v, q, a.out4);
}

// Local index of the feature corner of triangle q on a second step, or -1 (then it has a face
// point; on a first step every triangle has one).
__device__ __forceinline__ int feature_corner(const S3Args &a, int q) {
    if (a.odd) return -1;
    const int m = __ldg(a.fm + q);
    return m & 1 ? 0 : (m & 2 ? 1 : (m & 4 ? 2 : -1));
}

// The child corner that carries, on its own side, the unflipped edge of parent corner t (t >= 0):
// corner 0 of the child of t when t's triangle has a face point; else corner 1 of the last child
// (the edge b -> c) or corner 2 of the first (the edge c -> a) of its three-way split.
__device__ __forceinline__ int carry(const S3Args &a, int t) {
    const int q = t / 3, i = t - 3 * q, jq = feature_corner(a, q);
    if (jq < 0) return 3 * t;
    return i == (jq == 2 ? 0 : jq + 1) ? 3 * (3 * q + 2) + 1 : 3 * (3 * q) + 2;
}

// ternary cubic B-spline point of the feature edge a -> b nearer a: (beyond + 16 a + 10 b) / 27,
// beyond = the feature neighbour of a other than b, or the mirror 2 a - b at a curve end
__device__ __forceinline__ float3 third_point(const S3Args &a, int va, int vb, float3 pa, float3 pb) {
    const int4 ia = a.vi[va];
    float3 beyond;
    if (ia.x == 2) beyond = ldpv(a.P, ia.y == vb ? ia.z : ia.y, a.in4);
    else beyond = 2.0f * pa - pb;
    return (1.0f / 27.0f) * beyond + (16.0f / 27.0f) * pa + (10.0f / 27.0f) * pb;
}

__device__ __forceinline__ void push_crease(const S3Args &a, int u, int w) {
    const int i = atomicAdd(a.ccount, 1);
    if (i >= a.ccap) return;
    a.cverts[2 * i] = u;
    a.cverts[2 * i + 1] = w;
    a.csig[i] = INFINITY;
}

// 9 ints per triangle of the warp's 32 consecutive triangles (first r0, a multiple of 32): staged in
// shared memory and written as 16-byte stores (the warp's first int is 1152-byte aligned), clipped
// at n ints.
__device__ __forceinline__ void warp_rows9(int *dst, int r0, long long n, const int (&v)[9], int *sm) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 9; i++) sm[9 * lane + i] = v[i];
    __syncwarp();
    const long long g0 = 9LL * r0;
    int4 *o4 = reinterpret_cast<int4 *>(dst + g0);
    const int4 *s4 = reinterpret_cast<const int4 *>(sm);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int q = 32 * k + lane;
        if (q < 72) {
            const long long e = g0 + 4 * q;
            if (e + 4 <= n) {
                o4[q] = s4[q];
            } else {
                for (int t = 0; t < 4; t++)
                    if (e + t < n) dst[e + t] = sm[4 * q + t];
            }
        }
    }
    __syncwarp();
}

template <bool TOPO, bool EVAL>
__global__ void __launch_bounds__(kBlock) k_s3f_tri(S3Args a) {
    // with TOPO every lane of the warp takes part in the staged row stores (a lane past the last
    // triangle works on triangle 0 and its ints fall past the end); a failed status stops all
    const int r_in = blockIdx.x * blockDim.x + threadIdx.x;
    if (failed(a.status)) return;
    const bool live = r_in < a.F;
    if (!TOPO && !live) return;
    const int r = live ? r_in : 0;
    const int c = 3 * r, V = a.V;
    const int mask = __ldg(a.fm + r);
    int vv[3], tt[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        vv[j] = __ldg(a.fv + c + j);
        tt[j] = __ldg(a.tw + c + j);
    }
    const bool helpers = TOPO && a.twn;        // the child level is not the last one
    const int jf = a.odd ? -1 : (mask & 1 ? 0 : (mask & 2 ? 1 : (mask & 4 ? 2 : -1)));
    int fo[9], wo[9];
    if (jf < 0) {
        // a face point: every corner's child, its edge flipped unless a feature or (second
        // step) the triangle across has no face point
        bool flip[3];
#pragma unroll
        for (int j = 0; j < 3; j++) flip[j] = !((mask >> j) & 1) && (a.odd || feature_corner(a, tt[j] / 3) < 0);
        if (TOPO) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int jn = j == 2 ? 0 : j + 1, jp = j == 0 ? 2 : j - 1, t = tt[j];
                const bool fj = (mask >> j) & 1;
                fo[3 * j + 0] = vv[j];
                fo[3 * j + 1] = flip[j] ? V + t / 3 : vv[jn];
                fo[3 * j + 2] = V + r;
                if (live && fj && t >= 0 && c + j < t) push_crease(a, vv[j], vv[jn]);   // a kept crease edge
                if (!helpers) continue;
                wo[3 * j + 0] = flip[j] ? 3 * t_next(t) + 2 : (t < 0 ? t : carry(a, t));
                wo[3 * j + 1] = flip[j] ? 3 * t + 1 : 3 * (c + jn) + 2;
                wo[3 * j + 2] = flip[jp] ? 3 * tt[jp] : 3 * (c + jp) + 1;
                if (live) {
                    a.fmn[c + j] = fj ? 1 : 0;
                    if (__ldg(a.vc + vv[j]) == c + j) a.vcn[vv[j]] = 3 * (c + j);
                }
            }
            if (live && helpers) a.vcn[V + r] = 3 * c + 2;       // the face point: child 0, corner 2
        }
        if (EVAL && live) {
            const float3 p0 = ldpv(a.P, vv[0], a.in4), p1 = ldpv(a.P, vv[1], a.in4), p2 = ldpv(a.P, vv[2], a.in4);
            stpv(a.Pn, V + r, (1.0f / 3.0f) * (p0 + p1 + p2), a.out4);
        }
    } else {
        // second step, feature edge a -> b at corner jf, third vertex cc: split in three
        const int jb = jf == 2 ? 0 : jf + 1, jc = jf == 0 ? 2 : jf - 1;
        const int va = vv[jf], vb = vv[jb], vcc = vv[jc], tf = tt[jf];
        const int rank = -1 - tf;                              // a boundary edge's rank
        const int q1 = V + r, q2 = tf >= 0 ? V + tf / 3 : V + a.F + rank;
        if (TOPO) {
            fo[0] = va; fo[1] = q1; fo[2] = vcc;
            fo[3] = q1; fo[4] = q2; fo[5] = vcc;
            fo[6] = q2; fo[7] = vb; fo[8] = vcc;
            if (live && tf >= 0 && c + jf < tf) {               // the crease edge's three pieces
                push_crease(a, va, q1);
                push_crease(a, q1, q2);
                push_crease(a, q2, vb);
            }
            if (helpers) {
                const int rf = tf / 3;
                wo[0] = tf >= 0 ? 3 * (3 * rf + 2) : -1 - 3 * rank;
                wo[1] = 3 * (c + 1) + 2;
                wo[2] = carry(a, tt[jc]);
                wo[3] = tf >= 0 ? 3 * (3 * rf + 1) : -2 - 3 * rank;
                wo[4] = 3 * (c + 2) + 2;
                wo[5] = 3 * c + 1;
                wo[6] = tf >= 0 ? 3 * (3 * rf) : -3 - 3 * rank;
                wo[7] = carry(a, tt[jb]);
                wo[8] = 3 * (c + 1) + 1;
                if (live) {
                    a.fmn[c] = 1; a.fmn[c + 1] = 1; a.fmn[c + 2] = 1;
                    // carried corners: a at child 0 corner 0, b at child 2 corner 1, cc at child 0 corner 2
                    if (__ldg(a.vc + va) == c + jf) a.vcn[va] = 3 * c;
                    if (__ldg(a.vc + vb) == c + jb) a.vcn[vb] = 3 * (c + 2) + 1;
                    if (__ldg(a.vc + vcc) == c + jc) a.vcn[vcc] = 3 * c + 2;
                    a.vcn[q1] = 3 * c + 1;                     // q1: child 0, corner 1
                    if (tf < 0) a.vcn[q2] = 3 * (c + 1) + 1;   // a boundary q2: child 1, corner 1
                }
            }
        }
        if (EVAL && live) {
            const float3 pa = ldpv(a.P, va, a.in4), pb = ldpv(a.P, vb, a.in4);
            stpv(a.Pn, q1, third_point(a, va, vb, pa, pb), a.out4);
            if (tf < 0) stpv(a.Pn, q2, third_point(a, vb, va, pb, pa), a.out4);
        }
    }
    if (TOPO) {
        // the children's rows (and twins) of the warp's 32 triangles, 1152 contiguous bytes each
        __shared__ __align__(16) int srow[kBlock / 32][288];
        const int w = threadIdx.x >> 5, r0 = r_in - (int)(threadIdx.x & 31);
        warp_rows9(a.fvn, r0, 9LL * a.F, fo, srow[w]);
        if (helpers) warp_rows9(a.twn, r0, 9LL * a.F, wo, srow[w]);
    }
}

}  // namespace

}  // namespace alsub

namespace alsub {

void s3f_step(TopoImpl &T, int l, bool topo, const float *P, float *Pn, cudaStream_t s) {
    const LevelBuf &A = T.L[l];
    LevelBuf &B = T.L[l + 1];
    const bool ev = P != nullptr;
    if (!topo && !ev) return;
    const bool last = l + 1 == T.levels;
    S3Args a;
    a.l = l;
    a.V = (int)A.V;
    a.F = (int)A.F;
    a.odd = (l & 1) == 0;
    a.fv = A.fv; a.tw = A.tw; a.fm = A.fm;
    a.vc = l == 0 ? T.vc0 : A.vc;
    a.vi = T.s3_vi;
    a.P = P; a.Pn = Pn;
    a.in4 = l > 0;
    a.out4 = !last;
    a.fvn = B.fv;
    a.twn = last ? nullptr : B.tw;
    a.fmn = last ? nullptr : B.fm;
    a.vcn = last ? nullptr : B.vc;
    a.ccount = B.cr.xcount; a.cverts = B.cr.xverts; a.csig = B.cr.xsig;
    a.ccap = (int)B.cr.cap;
    a.status = T.status;
    if (l >= 1) {
        const LevelBuf &Pl = T.L[l - 1];
        a.pfv = Pl.fv; a.ptw = Pl.tw; a.pfm = Pl.fm;
        a.Vp = (int)Pl.V; a.Fp = (int)Pl.F;
        a.podd = ((l - 1) & 1) == 0;
    }
    if (l >= 2) {
        const LevelBuf &P2 = T.L[l - 2];
        a.p2tw = P2.tw; a.p2fm = P2.fm;
        a.V2 = (int)P2.V; a.F2 = (int)P2.F;
        a.p2odd = ((l - 2) & 1) == 0;
    }
    if (topo && B.cr.cap > 0) cudaMemsetAsync(B.cr.xcount, 0, sizeof(int), s);
    if (ev) {
        k_s3f_vert<true><<<grid_for(a.V), kBlock, 0, s>>>(a);
        T.launches += 1;
    }
    const unsigned g = grid_for(a.F);
    if (topo && ev) k_s3f_tri<true, true><<<g, kBlock, 0, s>>>(a);
    else if (topo) k_s3f_tri<true, false><<<g, kBlock, 0, s>>>(a);
    else k_s3f_tri<false, true><<<g, kBlock, 0, s>>>(a);
    T.launches += 1;
}

int s3f_export(TopoImpl &, int, cudaStream_t) {
    return 0;      // every level's crease list is written by the step that makes the level
}

}  // namespace alsub
