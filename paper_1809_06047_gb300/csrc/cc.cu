// Catmull-Clark refinement step (Sec. 3.2), one thread per parent face.
//
// Build (Fig. module_core, left): the child face table M_{l+1} (Sec. 3.2 "Topology refinement":
// corner x of face r becomes quad x = [v_x, |v|+|f|+e(x), |v|+r, |v|+|f|+e(prev x)]) and the
// per-corner E and F of level l+1, derived analytically from level l's:
//   child edge ids: the halves of parent edge e are 2e (at the owner's start vertex) and 2e+1;
//                   the edge from face point r to the edge point of corner c is 2E + c;
//   child twins:    corner 4c+0 <-> 4 next(tw(c)) + 3, 4c+1 <-> 4 next(c) + 2.
// On levels >= 1 every face is a quad (the reduced mesh matrix of Sec. 4.1), so M, E and F are
// int4 rows and corner x of face r is 4r + k.
//
// Eval (Fig. module_core, right), the mapped SpMVs fused into one pass:
//   face point   f = M^T P with val -> 1/c (Eq. spla_fp);
//   edge point   (p_k + p_l + f_r + f_s) / 4 for the corners that own their edge, with f_s
//                recomputed from the twin's face row instead of being re-read;
//   vertex point s1 + s2 + s3 = (1 - 2/n) p + 1/n^2 sum p_j + 1/n^2 sum f_j (Eq. pos_update in
//                its split form) gathered by the one corner designated for the vertex, walking the
//                ring x <- twin(prev(x)). The gather replaces the paper's atomic scatter (direct
//                mapped SpMV, Sec. 4.3) so that results are bit-reproducible.
//
// Open meshes (Sec. 3.2 "Boundaries", build and repair): corners without a twin carry twin -1 and
// the child rules keep it (a boundary edge splits into two boundary halves). The BND variants of
// the kernels skip every point whose stencil would cross the boundary (boundary edge points,
// boundary vertices); boundary_step then writes those from the level's boundary list.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

// L2 prefetch distance of the sibling kernel, in blocks (0 = none): each block asks the copy
// engine to bring the face rows (and the derived levels' ancestor rows) of the block this many
// indices ahead into L2, so that its first round trip starts from L2 instead of DRAM. One wave of
// a GB300 (152 SMs x 8 resident blocks); half a wave to two waves measured the same.
#ifndef ALSUB_SIB_PREFETCH
#define ALSUB_SIB_PREFETCH 1216
#endif
// The last step's face rows go out through shared memory, 512 contiguous bytes per store
// instruction (1), or straight from each lane, 64 bytes at a 64-byte stride (0).
#ifndef ALSUB_SIB_TOPO_SMEM
#define ALSUB_SIB_TOPO_SMEM 1
#endif
// Block size of the sibling kernel and the resident blocks per SM it is compiled for (register
// budget: 65536 / (block x blocks)).
#ifndef ALSUB_SIB_BLOCK
#define ALSUB_SIB_BLOCK 128
#endif
#ifndef ALSUB_SIB_MIN_BLOCKS
#define ALSUB_SIB_MIN_BLOCKS (1024 / ALSUB_SIB_BLOCK)
#endif

namespace alsub {

namespace {

struct CCArgs {
    int l;                        // parent level
    int V, F, E;                  // parent counts
    const int *fv, *ce, *tw;      // parent face table / edge ids / twins (flat, per corner)
    Level0 z;
    const float *P;               // parent positions
    float *Pn;                    // child positions
    int *fvn, *cen, *twn;         // child face table / edge ids / twins
    const int *pce, *ptw;         // edge ids / twins of the nearest stored ancestor level (l - 1 or
                                  // l - 2), used when level l's are not stored
    int Ep;                       // E of level l - 1
    int Epp;                      // E of level l - 2
    const int *twl[kMaxLevels];   // stored twins of every level (null where not stored)
    bool in4, out4;               // parent / child positions in padded float4 rows
    int *status;
    bool bnd;                     // the mesh is open (twins may be -1)
    bool rev;                     // sibling kernel: blocks take the faces from the end backwards
    int V0 = 0, F0 = 0;           // control-mesh counts and each control edge's owner corner (the
    const int *eo0 = nullptr;     // designated corners of level 1's vertices)
};

// Child twins across the halves of a parent edge (corner 0 and corner 3 of the children), or -1
// when the parent edge is a boundary edge.
template <bool BND>
__device__ __forceinline__ int twin_half0(int t) { return (BND && t < 0) ? -1 : 4 * quad_next(t) + 3; }
template <bool BND>
__device__ __forceinline__ int twin_half3(int t) { return (BND && t < 0) ? -1 : 4 * t; }

__device__ __forceinline__ float3 face_point_l0(const Level0 &z, const float *P, int g) {
    int s = __ldg(z.off + g), c = __ldg(z.off + g + 1) - s;
    float3 acc = f3(0.f, 0.f, 0.f);
    for (int j = 0; j < c; j++) acc += ldp(P, __ldg(z.fv + s + j));
    return (1.0f / (float)c) * acc;
}

// VERTS: the vertex points too (the ragged batch); else k_cc_l0_vert takes them after this kernel.
template <bool TOPO, bool HELP, bool EVAL, bool BND, bool VERTS = true>
__device__ __forceinline__ void cc_l0_body(const CCArgs &a, int r) {
    if (r >= a.F || failed(a.status)) return;
    const Level0 &z = a.z;
    const int s = __ldg(z.off + r), c = __ldg(z.off + r + 1) - s;
    const int VF = a.V + a.F, E2 = 2 * a.E;
    if (TOPO || HELP) {
        for (int j = 0; j < c; j++) {
            int x = s + j, p = (j == 0) ? s + c - 1 : x - 1;
            int ex = __ldg(z.ce + x), ep = __ldg(z.ce + p);
            if (TOPO) st4(a.fvn + 4 * (size_t)x, make_int4(__ldg(z.fv + x), VF + ex, a.V + r, VF + ep));
            if (HELP) {
                int ox = __ldg(z.own + x), op = __ldg(z.own + p);
                st4(a.cen + 4 * (size_t)x, make_int4(2 * ex + (ox ? 0 : 1), E2 + x, E2 + p, 2 * ep + (op ? 1 : 0)));
                const int tx = __ldg(z.tw + x), tp = __ldg(z.tw + p);
                st4(a.twn + 4 * (size_t)x, make_int4((BND && tx < 0) ? -1 : 4 * __ldg(z.nx + tx) + 3,
                                                     4 * __ldg(z.nx + x) + 2, 4 * p + 1, twin_half3<BND>(tp)));
            }
        }
    }
    if (EVAL) {
        const float *P = a.P;
        float3 fr = face_point_l0(z, P, r);
        stpv(a.Pn, a.V + r, fr, a.out4);
        for (int j = 0; j < c; j++) {
            int x = s + j;
            if (__ldg(z.own + x)) {
                int t = __ldg(z.tw + x);
                if (BND && t < 0) continue;          // boundary edge: repaired
                float3 fs = face_point_l0(z, P, __ldg(z.cf + t));
                float3 ep = 0.25f * (ldp(P, __ldg(z.fv + x)) + ldp(P, __ldg(z.fv + __ldg(z.nx + x))) + fr + fs);
                stpv(a.Pn, VF + __ldg(z.ce + x), ep, a.out4);
            }
        }
        for (int j = 0; VERTS && j < c; j++) {
            int x = s + j, v = __ldg(z.fv + x);
            if (__ldg(z.vc + v) != x) continue;
            int y = x, n = 0;
            float3 sp = f3(0.f, 0.f, 0.f), sf = f3(0.f, 0.f, 0.f);
            do {
                sf += face_point_l0(z, P, __ldg(z.cf + y));
                sp += ldp(P, __ldg(z.fv + __ldg(z.nx + y)));
                y = __ldg(z.rn + y);
                n++;
            } while ((!BND || y >= 0) && y != x && n < kMaxValence);
            if (BND && y < 0) continue;              // boundary vertex: repaired
            if (y != x) { set_status(a.status, ALSUB_ERR_UNSUPPORTED); continue; }
            float inv = 1.0f / (float)n;
            stpv(a.Pn, v, (1.0f - 2.0f * inv) * ldp(P, v) + (inv * inv) * (sp + sf), a.out4);
        }
    }
}

// VERTS: the vertex points too (the ragged batch); else k_cc_quad_vert takes them after this kernel.
template <bool TOPO, bool HELP, bool EVAL, bool BND, bool VERTS = true>
__device__ __forceinline__ void cc_quad_body(const CCArgs &a, int r) {
    if (r >= a.F || failed(a.status)) return;
    const int VF = a.V + a.F, E2 = 2 * a.E, c0 = 4 * r;
    const int4 v = ld4(a.fv + 4 * (size_t)r);
    const int4 e = ld4(a.ce + 4 * (size_t)r);
    int4 t = make_int4(0, 0, 0, 0);
    if (HELP || EVAL) t = ld4(a.tw + 4 * (size_t)r);
    if (TOPO) {
        int *o = a.fvn + 16 * (size_t)r;
        st4(o + 0, make_int4(v.x, VF + e.x, a.V + r, VF + e.w));
        st4(o + 4, make_int4(v.y, VF + e.y, a.V + r, VF + e.x));
        st4(o + 8, make_int4(v.z, VF + e.z, a.V + r, VF + e.y));
        st4(o + 12, make_int4(v.w, VF + e.w, a.V + r, VF + e.z));
    }
    if (HELP) {
        // corners 4r+0 and 4r+1 own their edges; 4r+2 and 4r+3 do not
        int *o = a.cen + 16 * (size_t)r;
        st4(o + 0, make_int4(2 * e.x, E2 + c0, E2 + c0 + 3, 2 * e.w));
        st4(o + 4, make_int4(2 * e.y, E2 + c0 + 1, E2 + c0, 2 * e.x + 1));
        st4(o + 8, make_int4(2 * e.z + 1, E2 + c0 + 2, E2 + c0 + 1, 2 * e.y + 1));
        st4(o + 12, make_int4(2 * e.w + 1, E2 + c0 + 3, E2 + c0 + 2, 2 * e.z));
        // corners 1 and 2 are interior edges of the parent face: only t.x and t.w can be -1
        int *w = a.twn + 16 * (size_t)r;
        st4(w + 0, make_int4(twin_half0<BND>(t.x), 4 * (c0 + 1) + 2, 4 * (c0 + 3) + 1, twin_half3<BND>(t.w)));
        st4(w + 4, make_int4(4 * quad_next(t.y) + 3, 4 * (c0 + 2) + 2, 4 * (c0 + 0) + 1, twin_half3<BND>(t.x)));
        st4(w + 8, make_int4(4 * quad_next(t.z) + 3, 4 * (c0 + 3) + 2, 4 * (c0 + 1) + 1, 4 * t.y));
        st4(w + 12, make_int4(twin_half0<BND>(t.w), 4 * (c0 + 0) + 2, 4 * (c0 + 2) + 1, 4 * t.z));
    }
    if (EVAL) {
        const float *P = a.P;
        const float3 p0 = ldpv(P, v.x, a.in4), p1 = ldpv(P, v.y, a.in4), p2 = ldpv(P, v.z, a.in4), p3 = ldpv(P, v.w, a.in4);
        const float3 fr = 0.25f * (p0 + p1 + p2 + p3);
        stpv(a.Pn, a.V + r, fr, a.out4);
        // edge points of the two owned edges (corners 4r and 4r+1)
        if (!BND || t.x >= 0) {
            int4 g = ld4(a.fv + 4 * (size_t)(t.x >> 2));
            float3 fs = 0.25f * (ldpv(P, g.x, a.in4) + ldpv(P, g.y, a.in4) + ldpv(P, g.z, a.in4) + ldpv(P, g.w, a.in4));
            stpv(a.Pn, VF + e.x, 0.25f * (p0 + p1 + fr + fs), a.out4);
        }
        {
            int4 g = ld4(a.fv + 4 * (size_t)(t.y >> 2));
            float3 fs = 0.25f * (ldpv(P, g.x, a.in4) + ldpv(P, g.y, a.in4) + ldpv(P, g.z, a.in4) + ldpv(P, g.w, a.in4));
            stpv(a.Pn, VF + e.y, 0.25f * (p1 + p2 + fr + fs), a.out4);
        }
        // vertex points gathered by designated corners (k = 3 is never designated)
#pragma unroll 1
        for (int k = 0; VERTS && k < 3; k++) {
            int x = c0 + k;
            if (!cc_vown(a.l, x, a.z)) continue;
            int y = x, n = 0;
            float3 sp = f3(0.f, 0.f, 0.f), sf = f3(0.f, 0.f, 0.f);
            do {
                int4 g = ld4(a.fv + 4 * (size_t)(y >> 2));
                float3 q0 = ldpv(P, g.x, a.in4), q1 = ldpv(P, g.y, a.in4), q2 = ldpv(P, g.z, a.in4), q3 = ldpv(P, g.w, a.in4);
                sf += 0.25f * (q0 + q1 + q2 + q3);
                int kk = (y + 1) & 3;
                sp += kk == 0 ? q0 : (kk == 1 ? q1 : (kk == 2 ? q2 : q3));
                y = __ldg(a.tw + quad_prev(y));
                n++;
            } while ((!BND || y >= 0) && y != x && n < kMaxValence);
            if (BND && y < 0) continue;              // boundary vertex: repaired
            if (y != x) { set_status(a.status, ALSUB_ERR_UNSUPPORTED); continue; }
            float inv = 1.0f / (float)n;
            int vk = comp(v, k);
            float3 pk = k == 0 ? p0 : (k == 1 ? p1 : p2);
            stpv(a.Pn, vk, (1.0f - 2.0f * inv) * pk + (inv * inv) * (sp + sf), a.out4);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Levels >= 2: the four children 4R..4R+3 of a parent quad R sit in four adjacent lanes. Child
// j is [a_j, b_j, c, b_{j-1}] with a_j the parent's corners, b_j its edge points and c its face
// point, so the group holds the 3 x 3 block of vertices in registers and shares them (and its
// face points) through width-4 shuffles instead of re-reading neighbour faces. The quad stencils
// below are the mapped SpMVs of Sec. 3.2 specialised to all-quad rows (Sec. 4.3 "Specializations":
// constant maps, reduced matrix):
//   edge point  3/8 (p_a + p_b) + 1/16 (the four far vertices of the two faces)  (Eq. 2, f_r, f_s
//               expanded), or (p_a + p_b + f_r + f_s) / 4 when both face points are in the group;
//   vertex      (1 - 7/(4n)) p + 3/(2n^2) sum next_g + 1/(4n^2) sum opp_g over the incident quads
//               g (Eq. pos_update with the face points expanded; n = 4 gives 1/64 [1 6 1; 6 36 6;
//               1 6 1]).
// The face point c and the edge points b_0, b_1 are gathered by the group itself (their rings are
// known analytically: the four siblings, and two siblings plus the two children of the twin
// corner); only vertices that existed on level l - 1 walk their ring through the twins.
// DERIVE: level l's per-corner edge ids and twins are not stored; they are derived from the
// parent level's (one int4 row per group), which saves writing and re-reading them on the last
// level.

__device__ __forceinline__ float3 shfl4(float3 v, int src) {
    return f3(__shfl_sync(0xffffffffu, v.x, src, 4), __shfl_sync(0xffffffffu, v.y, src, 4),
              __shfl_sync(0xffffffffu, v.z, src, 4));
}
__device__ __forceinline__ float3 sum4(float3 v) {
    v += f3(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1),
            __shfl_xor_sync(0xffffffffu, v.z, 1));
    v += f3(__shfl_xor_sync(0xffffffffu, v.x, 2), __shfl_xor_sync(0xffffffffu, v.y, 2),
            __shfl_xor_sync(0xffffffffu, v.z, 2));
    return v;
}

// The vertex at corner 4r (corner 0 of child r) existed on level l - 1; following x -> x / 4
// while x is a corner 0 walks back, with integer arithmetic only, to the level m where it was
// created, and tells which corner of that level designates it:
//   kind 1: the edge point of the level-(m-1) edge owned by corner c;
//   kind 2: the face point of the level-(m-1) face whose first corner is c;
//   kind 0: a vertex of the control mesh (c = one of its level-0 corners).
// Vertices created on levels >= 2 (all but a vanishing share on deep levels) are classified and
// get their four ring faces without touching memory apart from one stored twin; those created on
// levels 0 and 1 need the level-0 arrays and take the general path.
struct Birth {
    int m, k, c;
};
__device__ __forceinline__ Birth cc_descend(int l, int x) {
    int m = l;
    while (m > 0 && (x & 3) == 0) { x >>= 2; --m; }
    return Birth{m, m == 0 ? 0 : (x & 3), m == 0 ? x : (x >> 2)};
}
// designated on levels >= 2 (ALU only)
__device__ __forceinline__ int fast_kind(const Birth &b) {
    if (b.m < 2) return -1;
    if (b.k == 1 && (b.c & 3) < 2) return 1;
    if (b.k == 2 && (b.c & 3) == 0) return 2;
    return 0;   // not designated here
}

__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Face rows [f0, f0 + n) of a level with 4-int rows, clipped to its F faces (16-byte granules).
__device__ __forceinline__ void prefetch_rows(const int *rows, long long f0, long long n, long long F) {
    if (f0 < 0 || f0 >= F) return;
    if (f0 + n > F) n = F - f0;
    l2_prefetch(rows + 4 * f0, (unsigned)(16 * n));
}

// blk: the block's place in the order the blocks take the faces; its rows are prefetched that
// many blocks ahead in the same direction
template <bool TOPO, bool HELP, bool EVAL, int DERIVE, bool BND, bool RINGS>
__device__ __forceinline__ void cc_sib_body(const CCArgs &a, int r, int blk) {
    if (ALSUB_SIB_PREFETCH > 0 && threadIdx.x == 0) {
        const long long f0 = a.rev ? ((long long)blk - ALSUB_SIB_PREFETCH) * blockDim.x
                                   : ((long long)blk + ALSUB_SIB_PREFETCH) * blockDim.x;
        prefetch_rows(a.fv, f0, blockDim.x, a.F);
        if (DERIVE) {
            const int sh = 2 * DERIVE;        // ancestor rows: one per 4^DERIVE faces
            prefetch_rows(a.pce, f0 >> sh, (blockDim.x >> sh) + 1, (long long)a.F >> sh);
            prefetch_rows(a.ptw, f0 >> sh, (blockDim.x >> sh) + 1, (long long)a.F >> sh);
        }
    }
    if (failed(a.status)) return;
    const bool live = r < a.F;                  // F is a multiple of 4: groups are whole
    const int j = r & 3, R = r >> 2;
    const int VF = a.V + a.F, E2 = 2 * a.E, c0 = 4 * r;
    const int *__restrict__ fv = a.fv;
    const float *__restrict__ P = a.P;
    const Level0 &z = a.z;

    // ---- round trip 1: own row, adjacency rows, the twin an old vertex's ring needs
    const Birth b = cc_descend(a.l, c0);
    int fk = (EVAL && live) ? fast_kind(b) : 0;
    int tt = 0;
    if (fk == 1) tt = __ldg(a.twl[b.m - 1] + b.c);
    if (BND && fk == 1 && tt < 0) fk = 0;       // an edge point of a boundary edge: repaired
    int4 v = make_int4(0, 0, 0, 0), e = v, t = v;
    if (live) {
        v = ld4(fv + 4 * (size_t)r);
        if (DERIVE) {
            int4 pe, pt;                           // parent R's row of edge ids and twins
            if (DERIVE == 1) {
                pe = ld4(a.pce + 4 * (size_t)R);
                pt = ld4(a.ptw + 4 * (size_t)R);
            } else {
                // R is child k of grandparent G: the same child rules give R's rows from G's
                const int G = R >> 2, k = R & 3, kp = (k + 3) & 3, go = 4 * G + kp;
                const int4 ge = ld4(a.pce + 4 * (size_t)G), gt = ld4(a.ptw + 4 * (size_t)G);
                const int Epp2 = 2 * a.Epp;
                pe = make_int4(2 * comp(ge, k) + (k < 2 ? 0 : 1), Epp2 + R, Epp2 + go,
                               2 * comp(ge, kp) + (kp < 2 ? 1 : 0));
                pt = make_int4(twin_half0<BND>(comp(gt, k)), 4 * quad_next(R) + 2, 4 * go + 1,
                               twin_half3<BND>(comp(gt, kp)));
            }
            const int jp = (j + 3) & 3, po = 4 * R + jp;
            const int Ep2 = 2 * a.Ep;
            e = make_int4(2 * comp(pe, j) + (j < 2 ? 0 : 1), Ep2 + r, Ep2 + po,
                          2 * comp(pe, jp) + (jp < 2 ? 1 : 0));
            t = make_int4(twin_half0<BND>(comp(pt, j)), 4 * quad_next(r) + 2, 4 * po + 1,
                          twin_half3<BND>(comp(pt, jp)));
        } else {
            e = ld4(a.ce + 4 * (size_t)r);
            if (HELP || EVAL) t = ld4(a.tw + 4 * (size_t)r);
        }
    }
    if (EVAL) {
        // ---- round trip 2: own positions, rows of the two faces across edge (a_j, b_j),
        //      rows of the old vertex's ring
        const int s1 = t.x >> 2;                   // F1 = [a_j, y, z, b_j]
        const bool ob = BND && t.x < 0;            // (a_j, b_j) is a boundary edge: no F1, F2
        int4 g1 = make_int4(0, 0, 0, 0), g2 = g1, q0 = g1, q1 = g1;
        float3 pa = f3(0.f, 0.f, 0.f), pb = pa, pc = pa;
        if (live) {
            if (!ob) g1 = ld4(fv + 4 * (size_t)s1);
            if (j < 2 && !ob) g2 = ld4(fv + 4 * (size_t)quad_prev(s1));   // F2 = [a_{j+1}, b_j, z, w]
            pa = ldpv(P, v.x, true);
            pb = ldpv(P, v.y, true);
            if (j == 0) pc = ldpv(P, v.z, true);
        }
        if (fk > 0) {
            // The old vertex a_j is corner 0 of each of its four ring faces on level l (the ring
            // corners y on level m, shifted by sh): this face r (y0), F1 across (a_j, b_j), F3
            // across (d_j, a_j) = t.w's face, and the diagonal face F4. Rows r and F1 are loaded
            // already; F3 and F4 are the ones this vertex adds.
            const int sh = 2 * (a.l - b.m - 1);
            int y1, y2, y3;
            if (fk == 2) {
                y1 = 4 * b.c + 6; y2 = y1 + 4; y3 = y1 + 8;
            } else {
                y1 = 4 * quad_next(tt) + 3; y2 = 4 * tt + 1; y3 = 4 * quad_next(b.c) + 3;
            }
            const int f3 = t.w >> 2;
            const int z1 = y1 << sh, z2 = y2 << sh, z3 = y3 << sh;
            const int f4 = (z1 != s1 && z1 != f3) ? z1 : ((z2 != s1 && z2 != f3) ? z2 : z3);
            q0 = ld4(fv + 4 * (size_t)f3);
            q1 = ld4(fv + 4 * (size_t)f4);
        }
        pc = shfl4(pc, 0);                              // parent face point c
        const float3 pd = shfl4(pb, (j + 3) & 3);       // b_{j-1}
        const float3 fr = 0.25f * (pa + pb + pc + pd);  // face point of child j
        const float3 fn = shfl4(fr, (j + 1) & 3);       // face point of child j+1
        const float3 pan = shfl4(pa, (j + 1) & 3);      // a_{j+1}
        const float3 pbn = shfl4(pb, (j + 1) & 3);      // b_{j+1}
        const float3 sa = sum4(pa), sb = sum4(pb);
        if (live) {
            // ---- round trip 3: far vertices across (a_j, b_j), the old vertex's ring
            const float3 py = ob ? f3(0.f, 0.f, 0.f) : ldpv(P, g1.y, true);
            const float3 pz = ob ? f3(0.f, 0.f, 0.f) : ldpv(P, g1.z, true);
            const float3 pw = (j < 2 && !ob) ? ldpv(P, g2.w, true) : f3(0.f, 0.f, 0.f);
            float3 vp_old = f3(0.f, 0.f, 0.f);
            if (fk > 0) {
                // valence 4: (1 - 7/16) p + 3/32 sum next + 1/64 sum opp. Ring faces r = [a, b_j,
                // c, d_j], F1 = [a, y, z, b_j], F3 = [a, d_j, o3, u], F4 = [a, u, o4, y].
                const float3 pu = ldpv(P, q0.w, true), po3 = ldpv(P, q0.z, true), po4 = ldpv(P, q1.z, true);
                const float3 sn = (pb + pd) + (py + pu);
                const float3 so = (pc + pz) + (po3 + po4);
                vp_old = 0.5625f * pa + 0.09375f * sn + 0.015625f * so;
            }
            stpv(a.Pn, a.V + r, fr, a.out4);
            // interior edge (b_j, c) between children j and j+1
            stpv(a.Pn, VF + e.y, 0.25f * (pb + pc + fr + fn), a.out4);
            // edge (a_j, b_j) on the parent's edge, shared with F1
            if (!ob) stpv(a.Pn, VF + e.x, 0.375f * (pa + pb) + 0.0625f * (pc + pd + py + pz), a.out4);
            // face point c of the parent (valence 4): designated at child 0
            if (j == 0) stpv(a.Pn, v.z, 0.5625f * pc + 0.09375f * sb + 0.015625f * sa, a.out4);
            // edge point b_j of an owned parent edge (j < 2, valence 4): ring = children j, j+1, F1, F2
            if (j < 2 && !ob)
                stpv(a.Pn, v.y, 0.5625f * pb + 0.09375f * (pc + pa + pz + pan) + 0.015625f * (pd + py + pw + pbn),
                     a.out4);
            if (fk > 0) stpv(a.Pn, v.x, vp_old, a.out4);
            if (RINGS && fk < 0 && b.k != 3) {
                // created on level 0 or 1: designation and ring come from the level-0 record. Its
                // ring faces on level l are the descendants (index << sh) of the faces y listed
                // one level below the birth level, the vertex at their corner 0.
                const int sh = 2 * (a.l - b.m - 1);
                const int4 *rp = reinterpret_cast<const int4 *>(z.rec) + (size_t)(kRecInts / 4) * b.c;
                const int4 rh = __ldg(rp + ((b.m == 1 && b.k == 2) ? kRecFace / 4 : 0));
                float3 sn = f3(0.f, 0.f, 0.f), so = sn;
                int n = 0;
                bool walk = false, ok = true;
                int4 ra = make_int4(0, 0, 0, 0), rb = ra;
                if (b.m == 0) {
                    if (rh.x > 0) {                          // designated, closed ring of rh.x faces
                        n = rh.x;
                        ra = __ldg(rp + kRecRing / 4);
                        if (n > 4) rb = __ldg(rp + kRecRing / 4 + 1);
                    }
                    walk = rh.x == kRecLong;
                } else if (b.k == 1) {
                    if (rh.y >= 0) {                         // the owned edge's four ring faces
                        n = 4;
                        ra = make_int4(4 * b.c + 1, 4 * rh.z + 3, 4 * rh.y + 1, 4 * rh.w + 3);
                    }
                } else {
                    n = rh.x;                                // the first corner's face: its order
                }
                if (walk) {                                  // a long ring: walked
                    int y = b.c;
                    do {
                        const int4 q = ld4(fv + 4 * ((size_t)y << sh));
                        sn += ldpv(P, q.y, true);
                        so += ldpv(P, q.z, true);
                        y = __ldg(z.rn + y);
                        n++;
                    } while ((!BND || y >= 0) && y != b.c && n < kMaxValence);
                    ok = y == b.c;
                    if (BND && y < 0) n = 0;                 // a boundary vertex: repaired
                } else {
                    // four ring faces per round: their rows, then their positions
                    for (int i0 = 0; i0 < n; i0 += 4) {
                        int4 q[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int i = i0 + u;
                            const int y = (b.m == 1 && b.k == 2) ? 4 * (b.c + i) + 2
                                                                 : (i < 4 ? comp(ra, i) : comp(rb, i - 4));
                            if (i < n) q[u] = ld4(fv + 4 * ((size_t)y << sh));
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            if (i0 + u < n) {
                                sn += ldpv(P, q[u].y, true);
                                so += ldpv(P, q[u].z, true);
                            }
                        }
                    }
                }
                if (!ok) {
                    set_status(a.status, ALSUB_ERR_UNSUPPORTED);
                } else if (n > 0) {
                    const float inv = 1.0f / (float)n;
                    stpv(a.Pn, v.x, (1.0f - 1.75f * inv) * pa + (1.5f * inv * inv) * sn + (0.25f * inv * inv) * so,
                         a.out4);
                }
            }
        }
    }
    if (TOPO && ALSUB_SIB_TOPO_SMEM && DERIVE == 2) {
        // the warp's 32 faces write 128 consecutive int4 rows: staged in shared memory and
        // written back so that every store instruction covers 512 contiguous bytes (measured on
        // the last step only: 0.379 against 0.389 ms; the steps before it ran a little slower)
        __shared__ int4 stopo[ALSUB_SIB_BLOCK / 32][128];
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int4 *sb = stopo[w];
        sb[4 * lane + 0] = make_int4(v.x, VF + e.x, a.V + r, VF + e.w);
        sb[4 * lane + 1] = make_int4(v.y, VF + e.y, a.V + r, VF + e.x);
        sb[4 * lane + 2] = make_int4(v.z, VF + e.z, a.V + r, VF + e.y);
        sb[4 * lane + 3] = make_int4(v.w, VF + e.w, a.V + r, VF + e.z);
        __syncwarp();
        const int r0 = r - lane;
        int4 *o = reinterpret_cast<int4 *>(a.fvn) + 4 * (size_t)r0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int q = 32 * k + lane;
            if (r0 + (q >> 2) < a.F) o[q] = sb[q];
        }
    } else if (TOPO && live) {
        int *o = a.fvn + 16 * (size_t)r;
        st4(o + 0, make_int4(v.x, VF + e.x, a.V + r, VF + e.w));
        st4(o + 4, make_int4(v.y, VF + e.y, a.V + r, VF + e.x));
        st4(o + 8, make_int4(v.z, VF + e.z, a.V + r, VF + e.y));
        st4(o + 12, make_int4(v.w, VF + e.w, a.V + r, VF + e.z));
    }
    if (HELP && live) {
        int *o = a.cen + 16 * (size_t)r;
        st4(o + 0, make_int4(2 * e.x, E2 + c0, E2 + c0 + 3, 2 * e.w));
        st4(o + 4, make_int4(2 * e.y, E2 + c0 + 1, E2 + c0, 2 * e.x + 1));
        st4(o + 8, make_int4(2 * e.z + 1, E2 + c0 + 2, E2 + c0 + 1, 2 * e.y + 1));
        st4(o + 12, make_int4(2 * e.w + 1, E2 + c0 + 3, E2 + c0 + 2, 2 * e.z));
        int *w = a.twn + 16 * (size_t)r;
        st4(w + 0, make_int4(twin_half0<BND>(t.x), 4 * (c0 + 1) + 2, 4 * (c0 + 3) + 1, twin_half3<BND>(t.w)));
        st4(w + 4, make_int4(4 * quad_next(t.y) + 3, 4 * (c0 + 2) + 2, 4 * (c0 + 0) + 1, twin_half3<BND>(t.x)));
        st4(w + 8, make_int4(4 * quad_next(t.z) + 3, 4 * (c0 + 3) + 2, 4 * (c0 + 1) + 1, 4 * t.y));
        st4(w + 12, make_int4(twin_half0<BND>(t.w), 4 * (c0 + 0) + 2, 4 * (c0 + 2) + 1, 4 * t.z));
    }
}

template <bool TOPO, bool HELP, bool EVAL, bool BND>
__global__ void __launch_bounds__(kBlock) k_cc_l0(CCArgs a) {
    pdl_wait();
    pdl_trigger();
    cc_l0_body<TOPO, HELP, EVAL, BND, false>(a, blockIdx.x * blockDim.x + threadIdx.x);
}
// Level 0's vertex points, one thread per control vertex from its designated corner, after
// k_cc_l0: the ring's face points are read back from the level-1 positions k_cc_l0 stored (the
// same values the ring would recompute), the ring taken eight corners per round with the chain
// x <- twin(prev(x)) first. Sums in ring order, as cc_l0_body's.
template <bool BND>
__global__ void __launch_bounds__(kBlock) k_cc_l0_vert(CCArgs a) {
    pdl_wait();
    pdl_trigger();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V || failed(a.status)) return;
    const Level0 &z = a.z;
    const float *P = a.P;
    const int x = __ldg(z.vc + v);
    float3 sp = f3(0.f, 0.f, 0.f), sf = sp;
    int y = x, n = 0;
    bool done = false, open = false;
    while (!done && n < kMaxValence) {
        int ys[8];
        bool use[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            use[q] = !done;
            ys[q] = y;
            if (!done) {
                const int t = __ldg(z.rn + y);
                if (BND && t < 0) {
                    open = true;
                    done = true;
                } else {
                    y = t;
                    done = y == x || n + q + 1 >= kMaxValence;
                }
            }
        }
        int fq[8], wq[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            fq[q] = use[q] ? __ldg(z.cf + ys[q]) : 0;
            wq[q] = use[q] ? __ldg(z.fv + __ldg(z.nx + ys[q])) : 0;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (!use[q]) continue;
            sf += ldpv(a.Pn, a.V + fq[q], a.out4);
            sp += ldp(P, wq[q]);
            n++;
        }
    }
    if (BND && open) return;                   // boundary vertex: repaired
    if (y != x) { set_status(a.status, ALSUB_ERR_UNSUPPORTED); return; }
    const float inv = 1.0f / (float)n;
    stpv(a.Pn, v, (1.0f - 2.0f * inv) * ldp(P, v) + (inv * inv) * (sp + sf), a.out4);
}
template <bool TOPO, bool HELP, bool EVAL, bool BND>
__global__ void __launch_bounds__(kBlock) k_cc_quad(CCArgs a) {
    pdl_wait();
    pdl_trigger();
    cc_quad_body<TOPO, HELP, EVAL, BND, false>(a, blockIdx.x * blockDim.x + threadIdx.x);
}
// Level 1's vertex points, one thread per vertex after k_cc_quad, as k_cc_l0_vert does for level
// 0. The designated corner follows from the vertex's birth: a control vertex's is child 0 of its
// level-0 corner, a face point's corner 2 of its face's first child, an edge point's corner 1 of
// its owner corner's child. The ring's face points are read back from the level-2 positions
// k_cc_quad stored (the values cc_quad_body's ring recomputes, summed in the same order).
template <bool BND>
__global__ void __launch_bounds__(kBlock) k_cc_quad_vert(CCArgs a) {
    pdl_wait();
    pdl_trigger();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V || failed(a.status)) return;
    const Level0 &z = a.z;
    const float *P = a.P;
    int x;
    if (v < a.V0) x = 4 * __ldg(z.vc + v);
    else if (v < a.V0 + a.F0) x = 4 * __ldg(z.off + (v - a.V0)) + 2;
    else x = 4 * __ldg(a.eo0 + (v - a.V0 - a.F0)) + 1;
    float3 sp = f3(0.f, 0.f, 0.f), sf = sp;
    int y = x, n = 0;
    bool done = false, open = false;
    while (!done && n < kMaxValence) {
        int ys[8];
        bool use[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            use[q] = !done;
            ys[q] = y;
            if (!done) {
                const int t = __ldg(a.tw + quad_prev(y));
                if (BND && t < 0) {
                    open = true;
                    done = true;
                } else {
                    y = t;
                    done = y == x || n + q + 1 >= kMaxValence;
                }
            }
        }
        int wq[8];
#pragma unroll
        for (int q = 0; q < 8; q++) wq[q] = use[q] ? __ldg(a.fv + quad_next(ys[q])) : 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (!use[q]) continue;
            sf += ldpv(a.Pn, a.V + (ys[q] >> 2), a.out4);
            sp += ldpv(P, wq[q], a.in4);
            n++;
        }
    }
    if (BND && open) return;                   // boundary vertex: repaired
    if (y != x) { set_status(a.status, ALSUB_ERR_UNSUPPORTED); return; }
    const float inv = 1.0f / (float)n;
    stpv(a.Pn, v, (1.0f - 2.0f * inv) * ldpv(P, v, a.in4) + (inv * inv) * (sp + sf), a.out4);
}
// Vertices born on levels 0 and 1 are left to k_cc_ring01, which runs beside this kernel.
template <bool TOPO, bool HELP, bool EVAL, int DERIVE, bool BND>
__global__ void __launch_bounds__(ALSUB_SIB_BLOCK, ALSUB_SIB_MIN_BLOCKS) k_cc_sib(CCArgs a) {
    pdl_wait();
    pdl_trigger();
    const int blk = a.rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    cc_sib_body<TOPO, HELP, EVAL, DERIVE, BND, false>(a, blk * blockDim.x + threadIdx.x, blk);
}

// Vertex point, on a level l >= 2, of a vertex born on level m <= 1 whose ring faces on level l are
// the descendants (y << sh) of the faces y(i), i < n (the vertex at their corner 0, so the first
// row names it): (1 - 7/(4n)) p + 3/(2n^2) sum next + 1/(4n^2) sum opposite (Eq. pos_update on
// quads). Four ring faces per round trip pair (their rows, then their positions).
template <class Y>
__device__ __forceinline__ void ring_vertex(const CCArgs &a, int n, int sh, Y y) {
    const int *__restrict__ fv = a.fv;
    const float *__restrict__ P = a.P;
    float3 sn = f3(0.f, 0.f, 0.f), so = sn, p = sn;
    int vid = 0;
    for (int i0 = 0; i0 < n; i0 += 4) {
        int4 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (i0 + u < n) q[u] = ld4(fv + 4 * ((size_t)y(i0 + u) << sh));
        if (i0 == 0) {
            vid = q[0].x;
            p = ldpv(P, vid, true);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (i0 + u < n) {
                sn += ldpv(P, q[u].y, true);
                so += ldpv(P, q[u].z, true);
            }
        }
    }
    const float inv = 1.0f / (float)n;
    stpv(a.Pn, vid, (1.0f - 1.75f * inv) * p + (1.5f * inv * inv) * sn + (0.25f * inv * inv) * so, a.out4);
}

// Level l >= 2 step, the vertices the sibling kernel leaves out: those born on levels 0 and 1,
// one level-0 corner c per thread, from its ring record (Level0::rec): the control vertex c
// designates, the level-1 edge point of the edge c owns, the level-1 face point of the face whose
// first corner c is. Boundary vertices are skipped (the boundary repair writes them).
template <bool BND>
__global__ void __launch_bounds__(kBlock) k_cc_ring01(CCArgs a, int nnz0) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nnz0 || failed(a.status)) return;
    const int4 *rp = reinterpret_cast<const int4 *>(a.z.rec) + (size_t)(kRecInts / 4) * c;
    const int4 h0 = __ldg(rp), h1 = __ldg(rp + kRecFace / 4);
    const int sh1 = 2 * (a.l - 1), sh2 = 2 * (a.l - 2);
    if (h0.x > 0) {                                   // the control vertex: its ring corners
        const int4 ra = __ldg(rp + kRecRing / 4);
        const int4 rb = h0.x > 4 ? __ldg(rp + kRecRing / 4 + 1) : ra;
        ring_vertex(a, h0.x, sh1, [&](int i) { return i < 4 ? comp(ra, i) : comp(rb, i - 4); });
    } else if (h0.x == kRecLong) {                    // a longer ring: walked
        const int *__restrict__ fv = a.fv;
        float3 sn = f3(0.f, 0.f, 0.f), so = sn;
        int y = c, n = 0, vid = 0;
        do {
            const int4 q = ld4(fv + 4 * ((size_t)y << sh1));
            vid = q.x;
            sn += ldpv(a.P, q.y, true);
            so += ldpv(a.P, q.z, true);
            y = __ldg(a.z.rn + y);
            n++;
        } while (y >= 0 && y != c && n < kMaxValence);
        if (y != c) {
            if (!BND || y >= 0) set_status(a.status, ALSUB_ERR_UNSUPPORTED);
        } else {
            const float inv = 1.0f / (float)n;
            stpv(a.Pn, vid, (1.0f - 1.75f * inv) * ldpv(a.P, vid, true) + (1.5f * inv * inv) * sn +
                                (0.25f * inv * inv) * so, a.out4);
        }
    }
    if (h0.y >= 0) {                                  // the owned edge's four ring faces
        const int4 ra = make_int4(4 * c + 1, 4 * h0.z + 3, 4 * h0.y + 1, 4 * h0.w + 3);
        ring_vertex(a, 4, sh2, [&](int i) { return comp(ra, i); });
    }
    if (h1.x > 0)                                     // the face's order
        ring_vertex(a, h1.x, sh2, [&](int i) { return 4 * (c + i) + 2; });
}

// Boundary repair of step l (Sec. 3.2 "Boundaries"): entry i of level l's boundary list is the
// boundary edge a -> b, its successor the edge b -> c. It writes the edge point of (a, b) as the
// midpoint and the vertex point of b by Eq. CC_boundary, 3/4 p_b + 1/8 (p_a + p_c), over what the
// smooth step left there; every boundary edge and vertex has exactly one entry. With a child list,
// it also writes the two halves of (a, b) on level l + 1: a -> e at 2i (edge id 2e + 0 when the
// corner of (a, b) owns its edge, as level 0's boundary corners and levels >= 1's even entries,
// the corners 0 of their quads, do) and e -> b at 2i + 1, followed by the first half of b -> c.
__global__ void __launch_bounds__(kBlock) k_cc_bnd(int n, bool lvl0, const int *__restrict__ A,
                                                   const int *__restrict__ E, const int *__restrict__ S,
                                                   int *An, int *En, int *Sn, int V, int El, int VF,
                                                   const float *__restrict__ P, float *Pn, bool in4, bool out4,
                                                   int *status) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || failed(status)) return;
    auto clampi = [](int x, int hi) { return min(max(x, 0), hi - 1); };
    const int a = clampi(__ldg(A + i), V), e = clampi(__ldg(E + i), El), s1 = clampi(__ldg(S + i), n);
    const int b = clampi(__ldg(A + s1), V);
    if (P) {
        const int c = clampi(__ldg(A + clampi(__ldg(S + s1), n)), V);
        const float3 pa = ldpv(P, a, in4), pb = ldpv(P, b, in4), pc = ldpv(P, c, in4);
        stpv(Pn, VF + e, 0.5f * (pa + pb), out4);
        stpv(Pn, b, 0.75f * pb + 0.125f * (pa + pc), out4);
    }
    if (An) {
        const int h = (lvl0 || (i & 1) == 0) ? 0 : 1;
        An[2 * i] = a;
        En[2 * i] = 2 * e + h;
        Sn[2 * i] = 2 * i + 1;
        An[2 * i + 1] = VF + e;
        En[2 * i + 1] = 2 * e + 1 - h;
        Sn[2 * i + 1] = 2 * s1;
    }
}

// Ragged batches: the eval steps of many topologies at one level in one persistent launch per
// kernel class. The work list is the concatenation of every item's faces cut into tiles of
// blockDim.x faces (tile_begin[i] = first tile of item i, closed-form sizes); each CTA walks
// tiles with a grid stride and finds its item by binary search.
__device__ __forceinline__ int item_of(const int *__restrict__ tile_begin, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_begin + mid) <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int KIND>   // 0 level 0, 1 level 1, 2 levels >= 2, 3 / 4 levels >= 2 with E/F derived
                      // from the parent / grandparent level
__global__ void __launch_bounds__(512, 2) k_cc_batch(const CCArgs *__restrict__ items,
                                                     const int *__restrict__ tile_begin, int n, int tiles) {
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i = item_of(tile_begin, n, tile);
        const int r = (tile - __ldg(tile_begin + i)) * blockDim.x + threadIdx.x;
        const CCArgs &a = items[i];          // read in place: a copy would not fit in registers
        if (KIND == 0) cc_l0_body<false, false, true, false>(a, r);
        else if (KIND == 1) cc_quad_body<false, false, true, false>(a, r);
        else if (KIND == 2) cc_sib_body<false, false, true, 0, false, true>(a, r, blockIdx.x);
        else if (KIND == 3) cc_sib_body<false, false, true, 1, false, true>(a, r, blockIdx.x);
        else cc_sib_body<false, false, true, 2, false, true>(a, r, blockIdx.x);
    }
}

template <bool T, bool H, bool E, bool B>
void launch_b(const CCArgs &a, int derive, cudaStream_t s) {
    const unsigned g = grid_for(a.F, ALSUB_SIB_BLOCK);
    if (a.l == 0) {
        launch_pdl(k_cc_l0<T, H, E, B>, grid_for(a.F), kBlock, s, a);
        if (E) launch_pdl(k_cc_l0_vert<B>, grid_for(a.V), kBlock, s, a);
    }
    else if (a.l == 1) {
        launch_pdl(k_cc_quad<T, H, E, B>, grid_for(a.F), kBlock, s, a);
        if (E) launch_pdl(k_cc_quad_vert<B>, grid_for(a.V), kBlock, s, a);
    }
    else if (derive == 2) launch_pdl(k_cc_sib<T, false, E, 2, B>, g, ALSUB_SIB_BLOCK, s, a);
    else if (derive == 1) launch_pdl(k_cc_sib<T, false, E, 1, B>, g, ALSUB_SIB_BLOCK, s, a);
    else launch_pdl(k_cc_sib<T, H, E, 0, B>, g, ALSUB_SIB_BLOCK, s, a);
}
template <bool T, bool H, bool E>
void launch(const CCArgs &a, int derive, cudaStream_t s) {
    if (a.bnd) launch_b<T, H, E, true>(a, derive, s);
    else launch_b<T, H, E, false>(a, derive, s);
}

}  // namespace

namespace {

CCArgs make_args(TopoImpl &T, int l, const float *P, float *Pn, int *derive_out) {
    LevelBuf &A = T.L[l], &B = T.L[l + 1];
    CCArgs a;
    a.l = l;
    a.V = (int)A.V; a.F = (int)A.F; a.E = (int)A.E;
    a.fv = A.fv; a.ce = A.ce; a.tw = A.tw;
    a.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0, T.rn0,
                 T.rec0};
    a.P = P; a.Pn = Pn;
    a.fvn = B.fv; a.cen = B.ce; a.twn = B.tw;
    a.status = T.status;
    a.bnd = T.mesh->B > 0;
    a.V0 = (int)T.L[0].V;
    a.F0 = (int)T.L[0].F;
    a.eo0 = T.eo0;
    // consecutive steps take their faces in opposite orders, the last step from the end: a step
    // starts on the rows and positions its predecessor wrote last, which are still in L2
    a.rev = ((T.levels - 1 - l) & 1) == 0;
    a.in4 = l > 0;                     // only the caller's input level is packed xyz
    a.out4 = l + 1 < T.levels;         // and the caller's output level
    // a level >= 2 without stored edge ids / twins derives them from its parent level, or (level
    // >= 3 whose parent stores none either) from its grandparent
    int derive = 0;
    a.pce = nullptr; a.ptw = nullptr; a.Ep = 0; a.Epp = 0;
    if (l >= 2 && !A.helpers) {
        derive = T.L[l - 1].helpers ? 1 : 2;
        const LevelBuf &S = T.L[l - derive];
        a.pce = S.ce; a.ptw = S.tw;
        a.Ep = (int)T.L[l - 1].E;
        a.Epp = (int)T.L[l - 2].E;
    }
    for (int m = 0; m < kMaxLevels; m++) a.twl[m] = m <= T.levels && T.L[m].helpers ? T.L[m].tw : nullptr;
    *derive_out = derive;
    return a;
}

}  // namespace

void cc_step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s) {
    int derive = 0;
    CCArgs a = make_args(T, l, P, Pn, &derive);
    bool ev = P != nullptr;
    if (topo || ev) T.launches += 1;
    if (ev && l <= 1) T.launches += 1;           // k_cc_l0_vert, k_cc_quad_vert
    // levels >= 2: the vertices born on levels 0 and 1 go to k_cc_ring01, launched first on the
    // handle's ring stream beside the sibling kernel when it has one (forked and joined here, so
    // that its few blocks take SMs before the sibling kernel's grid fills them), else after it
    const bool rings = ev && l >= 2;
    const int nnz0 = T.mesh->nnz;
    auto launch_rings = [&](cudaStream_t rs) {
        if (a.bnd) k_cc_ring01<true><<<grid_for(nnz0), kBlock, 0, rs>>>(a, nnz0);
        else k_cc_ring01<false><<<grid_for(nnz0), kBlock, 0, rs>>>(a, nnz0);
        T.launches += 1;
    };
    const bool beside = rings && T.rside;
    if (beside) {
        cudaEventRecord(T.rfork, s);
        cudaStreamWaitEvent(T.rside, T.rfork, 0);
        launch_rings(T.rside);
        cudaEventRecord(T.rjoin, T.rside);
    }
    if (topo && helpers && ev) launch<true, true, true>(a, derive, s);
    else if (topo && helpers) launch<true, true, false>(a, derive, s);
    else if (topo && ev) launch<true, false, true>(a, derive, s);
    else if (topo) launch<true, false, false>(a, derive, s);
    else if (ev) launch<false, false, true>(a, derive, s);
    if (beside) cudaStreamWaitEvent(s, T.rjoin, 0);
    else if (rings) launch_rings(s);
    if (a.bnd) boundary_step(T, l, topo && l + 1 < T.levels, P, Pn, s);
}

void boundary_step(TopoImpl &T, int l, bool list, const float *P, float *Pn, cudaStream_t s) {
    const LevelBuf &A = T.L[l];
    if (A.B == 0 || (!list && !P)) return;
    LevelBuf *N = list ? &T.L[l + 1] : nullptr;
    // the edge point of edge e is |v| + |f| + e (Catmull-Clark) or |v| + e (Loop)
    const int first_edge_point = (int)(T.scheme == ALSUB_CATMULL_CLARK ? A.V + A.F : A.V);
    launch_pdl(k_cc_bnd, grid_for(A.B), kBlock, s, (int)A.B, l == 0, (const int *)A.bA, (const int *)A.bE,
               (const int *)A.bS, N ? N->bA : (int *)nullptr, N ? N->bE : (int *)nullptr, N ? N->bS : (int *)nullptr,
               (int)A.V, (int)A.E, first_edge_point, P, Pn, l > 0, l + 1 < T.levels, T.status);
    T.launches += 1;
}

std::vector<BatchClass> cc_batch_plan(const std::vector<EvalItem> &items, int block) {
    std::vector<CCArgs> args[5];
    std::vector<int> tiles[5];
    for (const EvalItem &it : items) {
        int derive = 0;
        CCArgs a = make_args(*it.T, it.l, it.P, it.Pn, &derive);
        a.rev = false;                      // the batch kernel walks its own tile list
        const int kind = it.l == 0 ? 0 : (it.l == 1 ? 1 : 2 + derive);
        if (tiles[kind].empty()) tiles[kind].push_back(0);
        args[kind].push_back(a);
        tiles[kind].push_back(tiles[kind].back() + (a.F + block - 1) / block);
    }
    std::vector<BatchClass> out;
    for (int k = 0; k < 5; k++) {
        if (args[k].empty()) continue;
        BatchClass c;
        c.kind = k;
        c.n = (int)args[k].size();
        c.tiles = tiles[k].back();
        if (cudaMalloc(&c.args, sizeof(CCArgs) * args[k].size()) != cudaSuccess ||
            cudaMalloc(&c.tile_begin, sizeof(int) * tiles[k].size()) != cudaSuccess) {
            cudaGetLastError();
            c.tiles = -1;  // allocation failed: caller reports OOM
            out.push_back(c);
            return out;
        }
        cudaMemcpy(c.args, args[k].data(), sizeof(CCArgs) * args[k].size(), cudaMemcpyHostToDevice);
        cudaMemcpy(c.tile_begin, tiles[k].data(), sizeof(int) * tiles[k].size(), cudaMemcpyHostToDevice);
        out.push_back(c);
    }
    return out;
}

void cc_batch_launch(const BatchClass &c, int block, int grid, cudaStream_t s) {
    const CCArgs *a = (const CCArgs *)c.args;
    const int g = std::max(1, std::min(grid, c.tiles));
    switch (c.kind) {
        case 0: k_cc_batch<0><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles); break;
        case 1: k_cc_batch<1><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles); break;
        case 2: k_cc_batch<2><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles); break;
        case 3: k_cc_batch<3><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles); break;
        default: k_cc_batch<4><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles); break;
    }
}

}  // namespace alsub
