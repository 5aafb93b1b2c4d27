// Loop (Appendix B) and sqrt(3) (Appendix A) refinement steps, one thread per parent triangle.
// Every level is a triangle mesh, so corner j of triangle r is 3r + j at every level (the reduced
// mesh matrix of Sec. 4.1 with an implicit column pointer).
//
// Loop. Build: triangle (v0, v1, v2) with edge ids e_j of corners j -> children
//   4r+0 = [v0, e0, e2], 4r+1 = [v1, e1, e0], 4r+2 = [v2, e2, e1], 4r+3 = [e0, e1, e2]
// (edge point of edge e has id |v| + e). Child edges: halves 2e (at the owner's start) and 2e+1,
// interior edge j (cutting corner j) 2E + 3r + j. Eval: edge point 3/8 (p_i + p_j) + 1/8 (p_k +
// p_l) with the opposite vertices read through G = the twin's third vertex (Appendix B, matrix G);
// vertex point (1 - n beta_n) p + beta_n sum p_j (Eq. loop_smooth) gathered around the ring.
//
// sqrt(3). Build: corner j of triangle r gives child 3r + j = [v_j, |v| + F(next, j), |v| + r]
// (Appendix A, "Topology refinement"; F(l,k) is the face across the corner's edge, i.e. the twin's
// face). Eval: face point = barycenter; vertex point (1 - alpha_n) p + alpha_n / n sum p_j
// (Eq. sqrt2, alpha_n of Eq. alpha).
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace alsub {

namespace {

__constant__ float c_loop_beta[kMaxValence + 1];
__constant__ float c_sqrt3_alpha[kMaxValence + 1];

struct TriArgs {
    int l;
    int V, F, E;
    const int *fv;
    TriLevel t;                   // edge ids / twins of level l (stored or derived)
    // level l - 1 (l >= 1; always stored): face table, edge ids, twins, vertex count
    const int *pfv = nullptr, *pce = nullptr, *ptw = nullptr;
    int Vp = 0;
    // every level's stored edge ids and twins (null where not stored) and edge counts
    const int *cel[kMaxLevels], *twl[kMaxLevels];
    int El[kMaxLevels];
    Level0 z;
    const float *P;
    float *Pn;
    int *fvn, *cen, *twn;
    bool in4, out4;               // parent / child positions in padded float4 rows
    bool rev = false;             // blocks take the triangles from the end backwards
    int *status;
};


// The face rows of a Loop / sqrt(3) step go out through shared memory, 512 contiguous bytes per
// store instruction (1), or straight from each lane, 48 / 36 bytes at that lane stride (0).
// Measured on the 128 x 128 tori: sqrt(3) L8 3.06 against 3.51 ms per step (its rows are 9 scalar
// ints); Loop L6 1.79 against 1.73 ms (its rows are three 16-byte stores already, and staging
// adds a spill).
#ifndef ALSUB_LOOP_TOPO_SMEM
#define ALSUB_LOOP_TOPO_SMEM 0
#endif
#ifndef ALSUB_SQRT3_TOPO_SMEM
#define ALSUB_SQRT3_TOPO_SMEM 1
#endif

// Levels >= 1 of a Loop step: the four children 4R..4R+3 of a parent triangle R sit in four
// adjacent lanes (F is a multiple of 4 and blocks hold whole groups), and a corner lane k < 3
// loads R's edge id and twin at corner k once for the group. The others come through width-4
// shuffles: a derived edge id of corner 2 (R's edge k - 1), and the positions of R's vertex v_k+1
// and edge point E_k+1, which are corners 0 and 1 of sibling k + 1 (its own row), so the parent's
// face table and those two ring positions are not read (1); or each lane loads them (0).
#ifndef ALSUB_LOOP_GROUP
#define ALSUB_LOOP_GROUP 1
#endif
// With the group, a level's edge ids come from the parent's by the child rules on every level
// >= 1, stored or not (1), or are read where the level stores them (0).
#ifndef ALSUB_LOOP_GROUP_IDS
#define ALSUB_LOOP_GROUP_IDS 1
#endif

__device__ __forceinline__ float3 shfl_down3(float3 v, int d) {
    return f3(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d),
              __shfl_down_sync(0xffffffffu, v.z, d));
}

__device__ __forceinline__ float3 shfl_g4(float3 v, int src) {
    return f3(__shfl_sync(0xffffffffu, v.x, src, 4), __shfl_sync(0xffffffffu, v.y, src, 4),
              __shfl_sync(0xffffffffu, v.z, src, 4));
}

// BND: an open mesh (Loop boundaries). Every stencil that would read across a corner without twin
// (-1) reads this triangle instead: the points it gives are the boundary edge points and boundary
// vertices, which the boundary step (cc.cu, boundary_step) writes afterwards from the level's
// boundary list; all other points never meet a boundary.
template <bool TOPO, bool HELP, bool EVAL, bool BND = false>
__device__ __forceinline__ void loop_body(const TriArgs &a, int r_in) {
    // with staged face rows every lane of the warp takes part in the stores (a lane past the end
    // works on face 0 and writes nothing); otherwise such a lane leaves at once
    constexpr bool STAGE = TOPO && ALSUB_LOOP_TOPO_SMEM;
    // a sibling group shuffles, so its lanes stay until the shuffles are done (a group is whole:
    // all four lanes live or none)
    const bool grp = ALSUB_LOOP_GROUP && a.l >= 1;
    const bool live = r_in < a.F && !failed(a.status);
    if (!STAGE && !grp && !live) return;
    const int r = live ? r_in : 0;
    const int c = 3 * r, V = a.V, E2 = 2 * a.E;
    const int R = r >> 2, k = r & 3;
    // the group's loads of parent R: edge id and twin at corner k (lane 3 repeats corner 2)
    const int kk = k < 3 ? k : 2;
    const int pek = grp ? __ldg(a.pce + 3 * R + kk) : 0;
    const int km = k == 0 ? 2 : k - 1;
    const int pem = grp ? __shfl_sync(0xffffffffu, pek, km, 4) : 0;    // R's edge k - 1
    int vv[3], ee[3], tt[3];
    bool ow[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        vv[j] = __ldg(a.fv + c + j);
        if (grp && (a.t.derive || ALSUB_LOOP_GROUP_IDS)) {
            // the child rules of the derived edge ids, with R's edges from the group
            const bool need = k != 3 && j != 1;
            const int q = j == 0 ? k : km;
            const bool own = need && loop_own_gi(a.t.lp, R, q, a.z);
            const int fromParent = 2 * (j == 0 ? pek : pem) + (j == 0 ? (own ? 0 : 1) : (own ? 1 : 0));
            const int interior = a.t.E2p + 3 * R + (k == 3 ? (j == 2 ? 0 : j + 1) : k);
            ee[j] = need ? fromParent : interior;
        } else {
            ee[j] = a.t.edge_gi(r, j);
        }
        // the eval of levels >= 1 reads its neighbours from the parent level: no twins needed
        tt[j] = (HELP || (EVAL && a.l == 0)) ? a.t.twin(c + j) : 0;
        ow[j] = loop_own_gi(a.l, r, j, a.z);
    }
    if (TOPO) {
        // the 12 ints of the four children, 48 bytes at 48 r
        const int4 q0 = make_int4(vv[0], V + ee[0], V + ee[2], vv[1]);
        const int4 q1 = make_int4(V + ee[1], V + ee[0], vv[2], V + ee[2]);
        const int4 q2 = make_int4(V + ee[1], V + ee[0], V + ee[1], V + ee[2]);
        if (STAGE) {
            // the warp's 32 faces own 96 consecutive int4: staged in shared memory and written
            // back 512 contiguous bytes per store instruction
            __shared__ int4 st[kBlock / 32][96];
            const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
            st[w][3 * lane + 0] = q0;
            st[w][3 * lane + 1] = q1;
            st[w][3 * lane + 2] = q2;
            __syncwarp();
            const int base = r_in - lane;
            int4 *o = reinterpret_cast<int4 *>(a.fvn) + 3 * (size_t)base;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = 32 * k + lane;
                if (base + q / 3 < a.F) o[q] = st[w][q];
            }
            if (!live && !grp) return;
        } else if (live) {
            int4 *o = reinterpret_cast<int4 *>(a.fvn + 12 * (size_t)r);
            o[0] = q0;
            o[1] = q1;
            o[2] = q2;
        }
    }
    if (HELP && live) {
        int oe[12], ot[12];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            int jp = j == 0 ? 2 : j - 1;
            oe[3 * j + 0] = 2 * ee[j] + (ow[j] ? 0 : 1);
            oe[3 * j + 1] = E2 + c + j;
            oe[3 * j + 2] = 2 * ee[jp] + (ow[jp] ? 1 : 0);
            int s = tt[j] / 3, i = tt[j] - 3 * s;
            ot[3 * j + 0] = (BND && tt[j] < 0) ? -1 : 3 * (4 * s + (i == 2 ? 0 : i + 1)) + 2;
            ot[3 * j + 1] = 3 * (4 * r + 3) + (j + 2) % 3;
            int s2 = tt[jp] / 3, i2 = tt[jp] - 3 * s2;
            ot[3 * j + 2] = (BND && tt[jp] < 0) ? -1 : 3 * (4 * s2 + i2) + 0;
            oe[9 + j] = E2 + c + (j + 1) % 3;
            ot[9 + j] = 3 * (4 * r + (j + 1) % 3) + 1;
        }
        int4 *pe = reinterpret_cast<int4 *>(a.cen + 12 * (size_t)r);
        int4 *pt = reinterpret_cast<int4 *>(a.twn + 12 * (size_t)r);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            pe[q] = make_int4(oe[4 * q], oe[4 * q + 1], oe[4 * q + 2], oe[4 * q + 3]);
            pt[q] = make_int4(ot[4 * q], ot[4 * q + 1], ot[4 * q + 2], ot[4 * q + 3]);
        }
    }
    if (EVAL) {
        const float *P = a.P;
        float3 p[3];
        // a group's centre lane gathers nothing
#pragma unroll
        for (int j = 0; j < 3; j++) p[j] = (grp && k == 3) ? f3(0.f, 0.f, 0.f) : ldpv(P, vv[j], a.in4);
        const int ptk = grp && a.l > 0 ? __ldg(a.ptw + 3 * R + kk) : 0;
        if (a.l == 0) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                if (!ow[j] || (BND && tt[j] < 0)) continue;      // a boundary edge: the boundary step
                int d = __ldg(a.fv + tri_prev(tt[j]));
                float3 ep = 0.375f * (p[j] + p[(j + 1) % 3]) + 0.125f * (p[(j + 2) % 3] + ldpv(P, d, a.in4));
                stpv(a.Pn, V + ee[j], ep, a.out4);
            }
#pragma unroll 1
            for (int j = 0; j < 3; j++) {
                int x = c + j;
                if (!loop_vown(a.l, x, a.z)) continue;
                int y = x, n = 0;
                float3 sp = f3(0.f, 0.f, 0.f);
                do {
                    sp += ldpv(P, __ldg(a.fv + tri_next(y)), a.in4);
                    y = a.t.twin(tri_prev(y));
                    n++;
                } while (y != x && n < kMaxValence && !(BND && y < 0));
                if (BND && y < 0) continue;                     // a boundary vertex: the boundary step
                if (y != x) { set_status(a.status, ALSUB_ERR_UNSUPPORTED); continue; }
                float beta = c_loop_beta[n];
                const float3 pj = j == 0 ? p[0] : (j == 1 ? p[1] : p[2]);   // constant indices: registers
                const int vj = j == 0 ? vv[0] : (j == 1 ? vv[1] : vv[2]);
                stpv(a.Pn, vj, (1.0f - (float)n * beta) * pj + beta * sp, a.out4);
            }
        } else {
            // Level l >= 1: this triangle is child k of triangle R of level l - 1, so its corner 0
            // is R's vertex v_k and its corner 1 the edge point E_k of R's edge k. Their rings on
            // level l are read from level l - 1, whose arrays are stored: the neighbours of v_k
            // are the edge points of its level-(l-1) edges (a walk of the stored parent ring);
            // those of E_k are v_k, v_k+1, E_k-1, E_k+1 and the two other edge points of the
            // triangle across edge k (valence 6).
            const int k1 = k >= 2 ? 0 : k + 1;
            // v_k+1 and E_k+1 are corners 0 and 1 of sibling k + 1
            const float3 gv = grp ? shfl_g4(p[0], k1) : f3(0.f, 0.f, 0.f);
            const float3 ge = grp ? shfl_g4(p[1], k1) : f3(0.f, 0.f, 0.f);
            if (!live) return;
            if (k < 3) {
                // The corner children own their corner-0 edge (the half v_k E_k of R's edge k) and
                // corner-1 edge (E_k E_k-1, inside R). Far vertices: across the half, E'_k2+1 of
                // the triangle R2 across edge k (twin 3 R2 + k2); across the inner edge, E_k+1.
                const int t0 = grp ? ptk : __ldg(a.ptw + 3 * R + k);
                const int t = (BND && t0 < 0) ? 3 * R + k : t0;    // across a boundary: R itself
                const int R2 = t / 3, k2 = t - 3 * R2;
                const int ea = a.Vp + __ldg(a.pce + 3 * R2 + (k2 == 2 ? 0 : k2 + 1));
                const float3 pen = grp ? ge : ldpv(P, a.Vp + __ldg(a.pce + 3 * R + k1), a.in4);
                const float3 pea = ldpv(P, ea, a.in4);
                stpv(a.Pn, V + ee[0], 0.375f * (p[0] + p[1]) + 0.125f * (p[2] + pea), a.out4);
                stpv(a.Pn, V + ee[1], 0.375f * (p[1] + p[2]) + 0.125f * (p[0] + pen), a.out4);
                if (loop_own_gi(a.l - 1, R, k, a.z)) {
                    // E_k: v_k, E_k-1 (this triangle), v_k+1, E_k+1, and E'_k2+1, E'_k2-1 across
                    const float3 pvn = grp ? gv : ldpv(P, __ldg(a.pfv + 3 * R + k1), a.in4);
                    const int eb = a.Vp + __ldg(a.pce + 3 * R2 + (k2 == 0 ? 2 : k2 - 1));
                    const float3 sp = (p[0] + p[2]) + (pvn + pen) + (pea + ldpv(P, eb, a.in4));
                    const float beta = c_loop_beta[6];
                    stpv(a.Pn, vv[1], (1.0f - 6.0f * beta) * p[1] + beta * sp, a.out4);
                }
            }
            if (k < 3 && loop_vown_gi(a.l, r, 0, a.z)) {
                // v_k = R's corner k. Follow it up while it is corner 0 of a corner child: it was
                // born on level m >= 1 as the midpoint of edge kb of triangle G of level m - 1
                // (valence 6), or is a control-mesh vertex (m = 0, any valence: walk the parent ring).
                int m = a.l - 1, x = 0, kb = 0, g = R, i = k;     // corner i of triangle g
                while (m > 0) {
                    const int j = g & 3;
                    if (i == 0 && j != 3) { i = j; g >>= 2; --m; continue; }
                    kb = j == 3 ? i : (i == 1 ? j : (j == 0 ? 2 : j - 1));
                    x = g >> 2;                      // G
                    break;
                }
                if (m > 0) {
                    // v's six edges on level m: the halves 2e, 2e + 1 of its birth edge e, and the
                    // interior edges kb, kb + 1 of G and kb2, kb2 + 1 of the triangle G2 across e;
                    // on each later level the half at v keeps v as an endpoint, its id doubling
                    // (plus one on the first split when v is not the edge owner's start).
                    const int G = x, c0 = 3 * G + kb;
                    const int eb = __ldg(a.cel[m - 1] + c0), t0 = __ldg(a.twl[m - 1] + c0);
                    const int t = (BND && t0 < 0) ? c0 : t0;       // born on the boundary: G itself
                    const int G2 = t / 3, kb2 = t - 3 * G2, I = 2 * a.El[m - 1];
                    const int id[6] = {2 * eb, 2 * eb + 1, I + 3 * G + kb, I + 3 * G + (kb == 2 ? 0 : kb + 1),
                                       I + 3 * G2 + kb2, I + 3 * G2 + (kb2 == 2 ? 0 : kb2 + 1)};
                    const int h[6] = {1, 1, 0, 1, 0, 1};
                    const int sh = a.l - 2 - m;          // levels after the first split
                    float3 sp = f3(0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 6; u++) {
                        const int e = m == a.l - 1 ? id[u] : ((2 * id[u] + h[u]) << sh);
                        sp += ldpv(P, a.Vp + e, a.in4);
                    }
                    const float beta = c_loop_beta[6];
                    stpv(a.Pn, vv[0], (1.0f - 6.0f * beta) * p[0] + beta * sp, a.out4);
                } else {
                    const int x0 = 3 * R + k;
                    int y = x0, n = 0;
                    float3 sp = f3(0.f, 0.f, 0.f);
                    do {
                        sp += ldpv(P, a.Vp + __ldg(a.pce + y), a.in4);
                        y = __ldg(a.ptw + tri_prev(y));
                        n++;
                    } while (y != x0 && n < kMaxValence && !(BND && y < 0));
                    if (BND && y < 0) {
                        // a boundary vertex: the boundary step
                    } else if (y != x0) {
                        set_status(a.status, ALSUB_ERR_UNSUPPORTED);
                    } else {
                        const float beta = c_loop_beta[n];
                        stpv(a.Pn, vv[0], (1.0f - (float)n * beta) * p[0] + beta * sp, a.out4);
                    }
                }
            }
        }
    }
}

// Levels >= 1 of a sqrt(3) step: the children 3T, 3T + 1, 3T + 2 of parent triangle T are
// adjacent lanes (F is a multiple of 3), and the ring of the face point f_T, designated at child
// 3T, is T's vertices and the face points across T's edges: corners 0 and 1 of the three
// children. Child 3T takes those of its siblings by shuffles when they are in its warp (lane <= 29),
// else it loads them (1); or it always loads them (0).
#ifndef ALSUB_SQRT3_GROUP
#define ALSUB_SQRT3_GROUP 1
#endif

template <bool TOPO, bool HELP, bool EVAL>
__device__ __forceinline__ void sqrt3_body(const TriArgs &a, int r_in) {
    constexpr bool STAGE = TOPO && ALSUB_SQRT3_TOPO_SMEM;   // as in loop_body
    // lanes stay until the shuffles of the siblings' positions are done
    const bool grp = ALSUB_SQRT3_GROUP && EVAL && a.l >= 1;
    const bool live = r_in < a.F && !failed(a.status);
    if (!STAGE && !grp && !live) return;
    const int r = live ? r_in : 0;
    const int c = 3 * r, V = a.V;
    int vv[3], tt[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        vv[j] = __ldg(a.fv + c + j);
        tt[j] = a.t.twin(c + j);
    }
    if (TOPO) {
        if (STAGE) {
            // the three children (9 ints, 36 bytes at 36 r): the warp's 288 consecutive ints are
            // staged in shared memory and written back as 72 int4, 512 contiguous bytes per store
            // instruction (the warp's first int is at 1152-byte alignment)
            __shared__ __align__(16) int st[kBlock / 32][288];
            const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                st[w][9 * lane + 3 * j + 0] = vv[j];
                st[w][9 * lane + 3 * j + 1] = V + tt[j] / 3;
                st[w][9 * lane + 3 * j + 2] = V + r;
            }
            __syncwarp();
            const long long g0 = 9LL * (r_in - lane), n = 9LL * a.F;
            int4 *o4 = reinterpret_cast<int4 *>(a.fvn + g0);
            const int4 *s4 = reinterpret_cast<const int4 *>(st[w]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = 32 * k + lane;
                if (q < 72) {
                    const long long e = g0 + 4 * q;
                    if (e + 4 <= n) {
                        o4[q] = s4[q];
                    } else {
                        for (int t = 0; t < 4; t++)
                            if (e + t < n) a.fvn[e + t] = st[w][4 * q + t];
                    }
                }
            }
            if (!live && !grp) return;
        } else if (live) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                int *o = a.fvn + 3 * (size_t)(c + j);
                o[0] = vv[j]; o[1] = V + tt[j] / 3; o[2] = V + r;
            }
        }
    }
    if (HELP && live) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            int *o = a.twn + 3 * (size_t)(c + j);
            int jp = j == 0 ? 2 : j - 1;
            o[0] = 3 * tri_next(tt[j]) + 2;
            o[1] = 3 * tt[j] + 1;
            o[2] = 3 * tt[jp] + 0;
        }
    }
    if (EVAL) {
        const float *P = a.P;
        float3 p[3];
#pragma unroll
        for (int j = 0; j < 3; j++) p[j] = ldpv(P, vv[j], a.in4);
        if (live) stpv(a.Pn, V + r, (1.0f / 3.0f) * (p[0] + p[1] + p[2]), a.out4);
        if (a.l == 0) {
#pragma unroll 1
            for (int j = 0; j < 3; j++) {
                int x = c + j;
                if (!sqrt3_vown(a.l, x, a.z)) continue;
                int y = x, n = 0;
                float3 sp = f3(0.f, 0.f, 0.f);
                do {
                    sp += ldpv(P, __ldg(a.fv + tri_next(y)), a.in4);
                    y = a.t.twin(tri_prev(y));
                    n++;
                } while (y != x && n < kMaxValence);
                if (y != x) { set_status(a.status, ALSUB_ERR_UNSUPPORTED); continue; }
                float al = c_sqrt3_alpha[n];
                const float3 pj = j == 0 ? p[0] : (j == 1 ? p[1] : p[2]);   // constant indices: registers
                const int vj = j == 0 ? vv[0] : (j == 1 ? vv[1] : vv[2]);
                stpv(a.Pn, vj, (1.0f - al) * pj + (al / (float)n) * sp, a.out4);
            }
        } else {
            // Level l >= 1: this triangle is the child of parent corner r, [v_r, f_F(r), f_T] with
            // T = r / 3. Rings on level l, read from the stored level l - 1: the old vertex v_r
            // neighbours the face points of its parent-level triangles (a walk of the parent
            // ring); f_T (designated at the child of T's corner 0) neighbours T's three vertices
            // and the face points of T's three neighbours (valence 6).
            // v_r = the vertex of parent corner r. Follow it up while it is corner 0 of a child:
            // the designated corner ends at corner 2 of the child of corner 3T of some triangle T
            // of level m - 1, i.e. v_r was born on level m >= 1 as T's face point (valence 6), or
            // is a control-mesh vertex (m = 0: its smallest corner designates it; walk the parent
            // ring). One descent serves the designation test and the ring.
            int m = a.l - 1, x = r;
            while (m > 0 && x % 3 == 0) { x /= 3; --m; }
            const bool des = live && (m > 0 ? (x % 3 == 2 && (x / 3) % 3 == 0)
                                             : __ldg(a.z.vc + __ldg(a.z.fv + x)) == x);
            if (des) {
                if (m > 0) {
                    // x = corner 2 of triangle g = x / 3 of level m, the child of corner g of
                    // triangle T = g / 3 of level m - 1. On level m, f_T lies in the children 3T + j
                    // of T's corners (corner 2) and in the children t = tw(3T + j) of the corners
                    // across (corner 1); on every later level in their corner-0 descendants (index
                    // x 3). Its neighbours on level l are the face points of these triangles on
                    // level l - 1.
                    const int T = x / 9;
                    float3 sp = f3(0.f, 0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 3; j++) {
                        const int t = __ldg(a.twl[m - 1] + 3 * T + j);
                        int X1 = 3 * T + j, X2 = t;                 // level m
                        if (m < a.l - 1) {
                            X1 = 3 * X1 + 2;                        // level m + 1
                            X2 = 3 * t + 1;
                            for (int q = m + 1; q < a.l - 1; q++) { X1 *= 3; X2 *= 3; }
                        }
                        sp += ldpv(P, a.Vp + X1, a.in4) + ldpv(P, a.Vp + X2, a.in4);
                    }
                    const float al = c_sqrt3_alpha[6];
                    stpv(a.Pn, vv[0], (1.0f - al) * p[0] + (al / 6.0f) * sp, a.out4);
                } else {
                    int y = r, n = 0;
                    float3 sp = f3(0.f, 0.f, 0.f);
                    do {
                        sp += ldpv(P, a.Vp + y / 3, a.in4);
                        y = __ldg(a.ptw + tri_prev(y));
                        n++;
                    } while (y != r && n < kMaxValence);
                    if (y != r) {
                        set_status(a.status, ALSUB_ERR_UNSUPPORTED);
                    } else {
                        const float al = c_sqrt3_alpha[n];
                        stpv(a.Pn, vv[0], (1.0f - al) * p[0] + (al / (float)n) * sp, a.out4);
                    }
                }
            }
            // corners 0 and 1 of the next two lanes (the siblings of a child 3T)
            const float3 s0a = grp ? shfl_down3(p[0], 1) : f3(0.f, 0.f, 0.f);
            const float3 s0b = grp ? shfl_down3(p[0], 2) : f3(0.f, 0.f, 0.f);
            const float3 s1a = grp ? shfl_down3(p[1], 1) : f3(0.f, 0.f, 0.f);
            const float3 s1b = grp ? shfl_down3(p[1], 2) : f3(0.f, 0.f, 0.f);
            if (live && r % 3 == 0) {
                // v_r = T's vertex 0 and f_F(r) = the face point across T's edge 0 are p[0], p[1];
                // T's vertices 1, 2 and the face points across its edges 1, 2 are corners 0 and 1
                // of children r + 1, r + 2
                float3 q1, q2, m1, m2;
                if (grp && (threadIdx.x & 31) <= 29) {
                    q1 = s0a; q2 = s0b; m1 = s1a; m2 = s1b;
                } else {
                    q1 = ldpv(P, __ldg(a.pfv + r + 1), a.in4);
                    q2 = ldpv(P, __ldg(a.pfv + r + 2), a.in4);
                    m1 = ldpv(P, a.Vp + __ldg(a.ptw + r + 1) / 3, a.in4);
                    m2 = ldpv(P, a.Vp + __ldg(a.ptw + r + 2) / 3, a.in4);
                }
                const float3 sp = (p[0] + p[1]) + (q1 + q2) + (m1 + m2);
                const float al = c_sqrt3_alpha[6];
                stpv(a.Pn, vv[2], (1.0f - al) * p[2] + (al / 6.0f) * sp, a.out4);
            }
        }
    }
}

TriArgs make_args(TopoImpl &T, int l, const float *P, float *Pn) {
    LevelBuf &A = T.L[l], &B = T.L[l + 1];
    TriArgs a;
    a.l = l;
    a.V = (int)A.V; a.F = (int)A.F; a.E = (int)A.E;
    a.fv = A.fv;
    a.t = tri_level(T, l);
    if (l >= 1) {
        const LevelBuf &Pl = T.L[l - 1];
        a.pfv = Pl.fv;
        a.pce = Pl.ce;
        a.ptw = Pl.tw;
        a.Vp = (int)Pl.V;
    }
    for (int m = 0; m < kMaxLevels; m++) {
        const bool st = m <= T.levels && T.L[m].helpers;
        a.cel[m] = st ? T.L[m].ce : nullptr;
        a.twl[m] = st ? T.L[m].tw : nullptr;
        a.El[m] = m <= T.levels ? (int)T.L[m].E : 0;
    }
    a.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0, T.rn0};
    a.P = P; a.Pn = Pn;
    a.fvn = B.fv; a.cen = B.ce; a.twn = B.tw;
    a.status = T.status;
    a.in4 = l > 0;
    a.out4 = l + 1 < T.levels;
    // consecutive steps take their triangles in opposite orders, the last step from the end: a
    // step starts on what its predecessor wrote last, still in L2
    a.rev = ((T.levels - 1 - l) & 1) == 0;
    return a;
}

// Resident 256-thread blocks per SM the Loop and sqrt(3) kernels are compiled for (register budget:
// 40 registers, measured faster than 5 blocks at 48 and than 8 blocks at 32 with spills).
#ifndef ALSUB_LOOP_MIN_BLOCKS
#define ALSUB_LOOP_MIN_BLOCKS 6
#endif
template <bool TOPO, bool HELP, bool EVAL, bool BND>
__global__ void __launch_bounds__(kBlock, ALSUB_LOOP_MIN_BLOCKS) k_loop(TriArgs a) {
    const unsigned blk = a.rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    loop_body<TOPO, HELP, EVAL, BND>(a, blk * blockDim.x + threadIdx.x);
}
template <bool TOPO, bool HELP, bool EVAL>
__global__ void __launch_bounds__(kBlock, ALSUB_LOOP_MIN_BLOCKS) k_sqrt3(TriArgs a) {
    const unsigned blk = a.rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    sqrt3_body<TOPO, HELP, EVAL>(a, blk * blockDim.x + threadIdx.x);
}

// Ragged batches (see the Catmull-Clark batch kernel): eval of many topologies at one level,
// tiles of blockDim.x triangles, grid-stride over tiles.
template <int KIND>   // 0 Loop, 1 sqrt(3)
__global__ void __launch_bounds__(512, 2) k_tri_batch(const TriArgs *__restrict__ items,
                                                      const int *__restrict__ tile_begin, int n, int tiles) {
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(tile_begin + mid) <= tile) lo = mid;
            else hi = mid - 1;
        }
        const int r = (tile - __ldg(tile_begin + lo)) * blockDim.x + threadIdx.x;
        const TriArgs &a = items[lo];          // read in place
        if (KIND == 0) loop_body<false, false, true>(a, r);
        else sqrt3_body<false, false, true>(a, r);
    }
}

}  // namespace

TriLevel tri_level(const TopoImpl &T, int l) {
    const LevelBuf &A = T.L[l];
    TriLevel t;
    t.sqrt3 = T.scheme == ALSUB_SQRT3;
    t.z = Level0{T.mesh->d_off, T.mesh->d_fv, T.cf0, T.nx0, T.pv0, T.L[0].tw, T.L[0].ce, T.own0, T.vc0, T.rn0};
    if (l >= 1) {                 // the parent's counts (the child rules need them either way)
        t.E2p = (int)(2 * T.L[l - 1].E);
        t.lp = l - 1;
    }
    if (A.helpers || l == 0) {
        t.ce = A.ce;
        t.tw = A.tw;
    } else {
        const LevelBuf &Pl = T.L[l - 1];
        t.derive = true;
        t.pce = Pl.ce;
        t.ptw = Pl.tw;
    }
    return t;
}

std::vector<BatchClass> tri_batch_plan(const std::vector<EvalItem> &items, int block) {
    std::vector<TriArgs> args[2];
    std::vector<int> tiles[2];
    for (const EvalItem &it : items) {
        TriArgs a = make_args(*it.T, it.l, it.P, it.Pn);
        a.rev = false;                      // the batch kernel walks its own tile list
        const int kind = it.T->scheme == ALSUB_LOOP ? 0 : 1;
        if (tiles[kind].empty()) tiles[kind].push_back(0);
        args[kind].push_back(a);
        tiles[kind].push_back(tiles[kind].back() + (a.F + block - 1) / block);
    }
    std::vector<BatchClass> out;
    for (int k = 0; k < 2; k++) {
        if (args[k].empty()) continue;
        BatchClass c;
        c.kind = k;
        c.n = (int)args[k].size();
        c.tiles = tiles[k].back();
        if (cudaMalloc(&c.args, sizeof(TriArgs) * args[k].size()) != cudaSuccess ||
            cudaMalloc(&c.tile_begin, sizeof(int) * tiles[k].size()) != cudaSuccess) {
            cudaGetLastError();
            c.tiles = -1;
            out.push_back(c);
            return out;
        }
        cudaMemcpy(c.args, args[k].data(), sizeof(TriArgs) * args[k].size(), cudaMemcpyHostToDevice);
        cudaMemcpy(c.tile_begin, tiles[k].data(), sizeof(int) * tiles[k].size(), cudaMemcpyHostToDevice);
        out.push_back(c);
    }
    return out;
}

void tri_batch_launch(const BatchClass &c, int block, int grid, cudaStream_t s) {
    const TriArgs *a = (const TriArgs *)c.args;
    const int g = grid < c.tiles ? (grid < 1 ? 1 : grid) : c.tiles;
    if (c.kind == 0) k_tri_batch<0><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles);
    else k_tri_batch<1><<<g, block, 0, s>>>(a, c.tile_begin, c.n, c.tiles);
}

void upload_weight_tables() {
    static std::once_flag once;
    std::call_once(once, [] {
        float beta[kMaxValence + 1], alpha[kMaxValence + 1];
        beta[0] = alpha[0] = 0.f;
        for (int n = 1; n <= kMaxValence; n++) {
            double t = 0.375 + 0.25 * cos(2.0 * M_PI / n);
            beta[n] = (float)((0.625 - t * t) / n);
            alpha[n] = (float)((4.0 - 2.0 * cos(2.0 * M_PI / n)) / 9.0);
        }
        cudaMemcpyToSymbol(c_loop_beta, beta, sizeof(beta));
        cudaMemcpyToSymbol(c_sqrt3_alpha, alpha, sizeof(alpha));
    });
}

template <bool B>
void launch_loop(const TriArgs &a, bool topo, bool helpers, bool ev, cudaStream_t s) {
    const unsigned g = grid_for(a.F);
    if (topo && helpers && ev) k_loop<true, true, true, B><<<g, kBlock, 0, s>>>(a);
    else if (topo && helpers) k_loop<true, true, false, B><<<g, kBlock, 0, s>>>(a);
    else if (topo && ev) k_loop<true, false, true, B><<<g, kBlock, 0, s>>>(a);
    else if (topo) k_loop<true, false, false, B><<<g, kBlock, 0, s>>>(a);
    else if (ev) k_loop<false, false, true, B><<<g, kBlock, 0, s>>>(a);
}

void loop_step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s) {
    TriArgs a = make_args(T, l, P, Pn);
    const bool ev = P != nullptr, bnd = T.mesh->B > 0;
    if (topo || ev) T.launches += 1;
    if (bnd) launch_loop<true>(a, topo, helpers, ev, s);
    else launch_loop<false>(a, topo, helpers, ev, s);
    // open mesh: boundary edge points and vertices, and the next level's boundary list
    if (bnd) boundary_step(T, l, topo && l + 1 < T.levels, P, Pn, s);
}

void sqrt3_step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s) {
    if (T.s3f) {
        s3f_step(T, l, topo, P, Pn, s);
        return;
    }
    TriArgs a = make_args(T, l, P, Pn);
    unsigned g = grid_for(a.F);
    bool ev = P != nullptr;
    if (topo || ev) T.launches += 1;
    if (topo && helpers && ev) k_sqrt3<true, true, true><<<g, kBlock, 0, s>>>(a);
    else if (topo && helpers) k_sqrt3<true, true, false><<<g, kBlock, 0, s>>>(a);
    else if (topo && ev) k_sqrt3<true, false, true><<<g, kBlock, 0, s>>>(a);
    else if (topo) k_sqrt3<true, false, false><<<g, kBlock, 0, s>>>(a);
    else if (ev) k_sqrt3<false, false, true><<<g, kBlock, 0, s>>>(a);
}

}  // namespace alsub
