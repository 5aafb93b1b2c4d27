// Host-side structures of libalsub and the launchers each .cu file provides.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "alsub.h"

namespace alsub {

// Sizes of carved sub-allocations, rounded up to 256 bytes.
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The crease matrix C_l of one level (Sec. 3.3) as a list of tagged edges. Level 0 keeps the
// input order; level l + 1 holds the two halves of entry i at 2i and 2i + 1, so entries whose
// sharpness decayed to 0 stay in the list as inert entries.
struct CreaseList {
    int *edge = nullptr;   // edge id at this level
    int *own = nullptr;    // corner that owns the edge
    float *sig = nullptr;  // sharpness (0 = inert)
    int *verts = nullptr;  // 2 endpoints per crease
    int *count = nullptr;  // number of entries (device int)
    long long cap = 0;     // host-side upper bound of the count
    // open-addressing table edge id -> sharpness bits (key -1 = empty), hmask + 1 = 2^k slots
    // probed in aligned pairs (bucket = (edge * 2654435761) >> (hshift + 1))
    int2 *tab = nullptr;
    int hmask = 0;
    int hshift = 32;       // 32 - k
    // per entry and end, in the order of verts (2i: verts[2i], 2i + 1: verts[2i + 1]), written
    // by the analysis and read by the fix: (k | designated << 16, sharpness sum bits, n1, n2)
    int4 *info = nullptr;
    // compacted copy (live creases only) written by crease_export
    int *xverts = nullptr;
    float *xsig = nullptr;
    int *xcount = nullptr;
};

// One level of the refined mesh. fv is the reduced mesh matrix (face table); ce and tw are the
// per-corner forms of the edge matrix E (Eq. CC_E) and face-adjacency matrix F (Eq. F).
struct LevelBuf {
    long long V = 0, F = 0, nnz = 0, E = 0;
    int *fv = nullptr;
    int *ce = nullptr;
    int *tw = nullptr;
    bool helpers = false;  // ce and tw are stored for this level
    // sqrt(3) with feature edges, levels below the last: per triangle, bit j set when corner j's
    // edge is a feature edge; per vertex, one of its outgoing corners (level 0: TopoImpl::vc0)
    unsigned char *fm = nullptr;
    int *vc = nullptr;
    CreaseList cr;
    // boundary list of an open Catmull-Clark or Loop mesh (levels below the last): entry i is a boundary
    // edge a -> b of this level with a = bA[i], edge id bE[i] and bS[i] = the entry of the next
    // boundary edge b -> c along the loop. Level 0 lists the boundary corners in any order;
    // level l + 1 holds the two halves of entry i at 2i (a -> edge point) and 2i + 1.
    long long B = 0;
    int *bA = nullptr, *bE = nullptr, *bS = nullptr;
};

// Where the device memory of a mesh, and of every handle made from it, comes from: the caller's
// allocator (alsub_mesh_create_ex) or, when `alloc` is null, CUDA's stream-ordered allocator.
struct DevAlloc {
    void *(*alloc)(size_t bytes, void *ctx, void *stream) = nullptr;
    void (*free)(void *ptr, void *ctx, void *stream) = nullptr;
    void *ctx = nullptr;
};
// Stream-ordered allocation of `bytes` on `s` (cudaSuccess, or cudaErrorMemoryAllocation with *p
// null; no CUDA error is left pending) and its release after the work enqueued on `s`.
cudaError_t dev_malloc(const DevAlloc &A, void **p, size_t bytes, cudaStream_t s);
void dev_free(const DevAlloc &A, void *p, cudaStream_t s);
template <class T>
cudaError_t dev_malloc(const DevAlloc &A, T **p, size_t bytes, cudaStream_t s) {
    return dev_malloc(A, reinterpret_cast<void **>(p), bytes, s);
}

struct MeshImpl {
    alsub_scheme scheme;
    int V = 0, F = 0, nnz = 0, K = 0;
    float sigma_max = 0.f;     // largest input sharpness (inf allowed)
    int *d_off = nullptr;      // F + 1
    int *d_fv = nullptr;       // nnz
    int *d_cv = nullptr;       // 2K
    float *d_cs = nullptr;     // K
    int B = 0;                 // boundary edges (Catmull-Clark open meshes)
    int *d_vmap = nullptr;     // extracted meshes (selective subdivision): kept vertex -> source vertex
    int *d_fmap = nullptr;     //                                           kept face -> source face
    const void *src_topo = nullptr;   // extracted meshes: the topology and level they were taken
    int src_level = -1;               // from (identity only: it is never dereferenced)
    void *d_block = nullptr;   // one allocation holding d_off, d_fv, d_cv, d_cs and d_status (or
                               // null: those are allocated one by one)
    int *d_status = nullptr;   // checks of the mesh that run on the device (the boundary edge count
                               // a caller stated): 0, or the error each level-0 build starts from
    cudaStream_t stream = nullptr;
    DevAlloc alloc;            // every device array of the mesh and of its handles
};

// A captured refine call: replayed while its pointers (and timing mode) stay the same.
struct CallGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *P0 = nullptr, *PL = nullptr, *scratch = nullptr;
    bool timed = false;
    long long launches = 0;                 // kernels one replay runs
    std::vector<cudaGraphNode_t> marks;     // timing event-record nodes, by mark index
    unsigned long long used = 0;            // last use (LRU)
};

// Open-addressing table of the level-0 directed edges (a, b) -> corner, 2^k slots (key ~0 = empty).
struct DirTable {
    unsigned long long *key = nullptr;
    int *val = nullptr;
    unsigned mask = 0;
};

struct TopoImpl {
    MeshImpl *mesh = nullptr;
    DevAlloc alloc;              // the mesh's allocator, copied: the arrays are released with it
                                 // even when the mesh is destroyed first
    alsub_scheme scheme;
    int levels = 0;
    std::vector<LevelBuf> L;     // levels + 1
    // level-0 adjacency
    int *cf0 = nullptr, *nx0 = nullptr, *pv0 = nullptr, *own0 = nullptr, *vc0 = nullptr;
    int *eo0 = nullptr, *deg = nullptr, *rn0 = nullptr;   // rn0: twin(prev(x)), the ring step
    // Catmull-Clark: the rings of the vertices born on levels 0 and 1, per level-0 corner c, 16
    // ints (see kRec* in common.cuh), read by the steps of levels >= 2 instead of walking them
    int *rec0 = nullptr;
    // sqrt(3) with feature edges (boundary edges, infinitely sharp creases): the general path of
    // sqrt3f.cu, with per-vertex scratch for the largest level a step starts from
    bool s3f = false;
    int4 *s3_vi = nullptr;       // feature valency and feature neighbours of every vertex
    DirTable dir;
    int *eid = nullptr, *e0count = nullptr;
    int *bcount = nullptr;       // boundary corners found on level 0
    int *status = nullptr;       // latched device error
    // temporaries
    void *scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    int *flags = nullptr;        // max(nnz0, E0, 2 * max crease cap) ints
    int *pos = nullptr;          // scan output of flags, same size
    float *scratch = nullptr;    // intermediate positions (two levels)
    size_t scratch_bytes = 0;
    std::vector<void *> allocs;  // everything above, freed on destroy
    size_t bytes = 0;            // device bytes in allocs
    bool dry = false;            // size the allocations without making them (alsub_plan_bytes)
    char *arena = nullptr;       // the handle's arrays are carved from one allocation
    size_t arena_off = 0, arena_size = 0;
    cudaStream_t stream = nullptr;
    bool built = false;
    // live timing (alsub_topology_set_timing) and launch count
    int tcap = 0;
    int tcalls = 0;
    std::vector<cudaEvent_t> tev;           // (tcap + 1) slots of levels + 2 events; the last
                                            // slot absorbs calls beyond the capacity
    long long launches = 0;
    // CUDA graphs of alsub_refine_vertices ([0]) and alsub_subdivide ([1]) calls, a few per kind
    static constexpr int kGraphs = 4;
    CallGraph graphs[2][kGraphs];
    unsigned long long graph_clock = 0;
    const void *last[2][3] = {};            // pointers of the previous call of each kind: a call is
                                            // captured the second time its arguments repeat
    cudaStream_t cap = nullptr;             // private stream the calls are captured on
    bool capturing = false;
    // side branch of alsub_subdivide: the crease analysis of level l runs beside the level's
    // build + eval step (fork after the step that built level l, join before the crease fix)
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t> fork_ev, join_ev;   // levels + 1 each
    cudaEvent_t ring_ev = nullptr;               // the ring records of level 0 are written
    // Catmull-Clark levels >= 2: the stream the vertices born on levels 0 and 1 are refined on,
    // beside the step's main kernel (fork and join events reused level after level)
    cudaStream_t rside = nullptr;
    cudaEvent_t rfork = nullptr, rjoin = nullptr;
    // hierarchical edits (alsub_topology_set_edits): per level, offsets added to its vertices after
    // the level has been refined
    struct LevelEdits {
        int n = 0;
        int *vid = nullptr;
        float *off = nullptr;
    };
    std::vector<LevelEdits> edits;           // levels + 1 (level 0 unused)
    // alsub_subdivide_host: upload + eval stream, download stream, device input, two device
    // outputs, two page-locked input stagings and their events (indexed by call parity)
    struct HostIO {
        cudaStream_t cs = nullptr, ds = nullptr;
        float *dP0 = nullptr, *dPL[2] = {nullptr, nullptr}, *hP0[2] = {nullptr, nullptr};
        cudaEvent_t up[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
        unsigned long long calls = 0;
        bool ready = false;
    } io;
};

// ---------------------------------------------------------------- launchers

// Exclusive scan of n ints (elements at index >= *n_dev read as 0 when n_dev is given); the
// total goes to *total when total is not null. tmp must hold scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(long long n);
int scan_exclusive(const int *in, int *out, long long n, int *total, const int *n_dev, void *tmp,
                   cudaStream_t s);  // returns the number of kernels launched
// Same over int32 counts into int64 offsets (operator row pointers).
int scan_exclusive64(const int *in, long long *out, long long n, long long *total, void *tmp,
                     cudaStream_t s);

// Level 0: corner maps, twins, ownership, edge numbering, ring steps.
void level0_build(TopoImpl &T, cudaStream_t s);
// Level 0's per-vertex checks (in some face, valence, single fan); only sets the status word.
void level0_validate(TopoImpl &T, cudaStream_t s);
// Level 0's crease list and hash table (needs level0_build's arrays).
void level0_creases(TopoImpl &T, cudaStream_t s);
// Boundary edges of a Catmull-Clark control mesh (corners whose reverse edge is in no face) and
// whether a crease touches a boundary vertex; synchronises `s`.
alsub_status mesh_boundary_scan(MeshImpl &M, cudaStream_t s, long long *B, bool *crease_at_boundary);
// The same scan with the count a caller stated (M.B = B_stated) checked on the device instead of
// read back: M.d_status becomes UNSUPPORTED (a crease touches a boundary vertex), NONMANIFOLD
// (nnz + B odd) or INVALID_ARG (another count than B_stated). Nothing is synchronised.
alsub_status mesh_boundary_check(MeshImpl &M, cudaStream_t s, long long B_stated);
// Vertices on a boundary edge (flag 1) of a face table (off == nullptr: uniform quads).
alsub_status level_boundary_flags(int V, int F, long long nnz, const int *off, const int *fv, int *flag,
                                  const DevAlloc &A, cudaStream_t s);
// Extraction of selective subdivision (Sec. 3.4) from level `level` of a built topology into a new
// mesh (device arrays, maps, creases; B not yet set); synchronises `s`.
alsub_status extract_level(TopoImpl &T, int level, const unsigned char *mask, int rings, cudaStream_t s,
                           MeshImpl &out);
// The hierarchical edits of level k (1 .. levels) added to its freshly refined positions `out`.
void apply_edits(TopoImpl &T, int k, float *out, cudaStream_t s);
// P' = X P: rows vmap[i] of P into row i of out (xyz rows).
void gather_rows(int n, const int *vmap, const float *P, float *out, cudaStream_t s);
// Mesh reordering (Sec. 4.5): RCM on the graph of the mesh Laplacian, faces sorted by their least
// new vertex; fills `out` (arrays, maps, counts) on `s`, which it synchronises once per
// breadth-first level. *levels_out: breadth-first levels over all components.
alsub_status reorder_mesh(const MeshImpl &M, cudaStream_t s, MeshImpl &out, int *levels_out);
// Boundary repair of one Catmull-Clark or Loop step (Sec. 3.2 "Boundaries", Fig.
// module_boundary; Loop takes the same rules): with positions, overwrite the boundary edge points
// (midpoints) and boundary vertices (Eq. CC_boundary) of level l + 1; with `list`, write level
// l + 1's boundary list (the halves' edge ids follow both schemes' rule: the half at the owner
// corner's start is 2e, where the owner of a boundary half is its one corner on even entries).
void boundary_step(TopoImpl &T, int l, bool list, const float *P, float *Pn, cudaStream_t s);

// One refinement step from level l to l + 1. topo: emit the child face table; helpers: emit the
// child's per-corner edge ids and twins; P/Pn: parent/child positions (null = no vertex eval).
void cc_step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s);
void loop_step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s);
void sqrt3_step(TopoImpl &T, int l, bool topo, bool helpers, const float *P, float *Pn, cudaStream_t s);

// sqrt(3) with feature edges (sqrt3f.cu). s3f_level0: after level0_build, the boundary corners'
// twins become -1 - rank (rank in corner order) and the per-corner feature flags of level 0 are set
// and crease list (boundary edges, infinitely sharp creases). s3f_step: one step l -> l + 1
// (topology and/or positions). s3f_export: nothing to do (the steps keep every level's crease list
// current; returns the launches).
void s3f_level0(TopoImpl &T, cudaStream_t s);
// The sqrt(3) feature path's weight table into constant memory (once; before any capture).
void s3f_upload_tables();
void s3f_step(TopoImpl &T, int l, bool topo, const float *P, float *Pn, cudaStream_t s);
int s3f_export(TopoImpl &T, int l, cudaStream_t s);

// True when level l has a crease list to analyse and fix.
bool crease_alive(const TopoImpl &T, int l);
// Analysis of level l's creases (crease valency and sharpness sum at both ends from the ring
// walks, kept per entry for crease_fix); with `inherit`, also the crease list and hash table of
// level l + 1 (Sec. 3.3). Needs level l's adjacency, not positions.
void crease_analyse(TopoImpl &T, int l, bool inherit, cudaStream_t s);
// Overwrite the crease edge points and crease vertices of level l + 1 (Fig. module_creases) from
// the stored analysis of level l, after the smooth eval of the level.
void crease_fix(TopoImpl &T, int l, const float *P, float *Pn, cudaStream_t s);
void crease_table_clear(const CreaseList &C, cudaStream_t s);
// Compact level l's list (drop the inert zero-sharpness entries) into its x* arrays; returns the
// number of kernels launched.
int crease_export(TopoImpl &T, int l, cudaStream_t s);

// Device-side constant tables (Loop beta_n, sqrt(3) alpha_n) filled once per process.
void upload_weight_tables();

// Record `msg` as the calling thread's last error and return `s`.
alsub_status report(alsub_status s, const char *msg);

// ---- ragged batches: the eval steps of many topologies at one level in one launch per class
struct EvalItem {
    TopoImpl *T;
    int l;                 // level whose step is evaluated (l -> l + 1)
    const float *P;        // level-l positions
    float *Pn;             // level-(l+1) positions
};
struct BatchClass {
    int kind = 0;          // kernel variant
    int n = 0;             // items
    int tiles = 0;         // total tiles (blockDim.x faces each); -1 when the plan failed
    void *args = nullptr;  // device array of per-item kernel arguments (cudaMalloc)
    int *tile_begin = nullptr;  // n + 1 tile offsets (cudaMalloc)
};
std::vector<BatchClass> cc_batch_plan(const std::vector<EvalItem> &items, int block);
void cc_batch_launch(const BatchClass &c, int block, int grid, cudaStream_t s);
std::vector<BatchClass> tri_batch_plan(const std::vector<EvalItem> &items, int block);
void tri_batch_launch(const BatchClass &c, int block, int grid, cudaStream_t s);

// Edge ids and twins of a Loop / sqrt(3) level, stored or derived from the parent level's
// (TriLevel is defined with the device helpers).
struct TriLevel;
TriLevel tri_level(const TopoImpl &T, int l);

// One vertex refinement of a built topology as alsub_refine_vertices makes it (a repeated call
// replays a captured graph); `scratch` holds the intermediate levels (null: the handle's own).
alsub_status refine_call(TopoImpl &T, const float *P0, float *PL, void *scratch, cudaStream_t s);
// One vertex refinement of a built topology, its kernels launched directly on `s`: no graph is
// captured or replayed and no stream or event is made (the graph cache is left as it is).
alsub_status refine_direct(TopoImpl &T, const float *P0, float *PL, void *scratch, cudaStream_t s);
// Matrix-free adjoint of the Catmull-Clark steps of a closed mesh (g_l = R_l^T g_{l+1} gathered per
// coarse vertex). Per level, computed once from the topology (which must store the level's edge
// ids and twins): each vertex's coefficients (float4), designated corner and (levels >= 1) the
// slot of each corner's contribution, and on a level with creases each edge's min(sigma, 1). adjoint_step gathers one level
// (G: level l + 1, g: level l; float4 rows or packed xyz; part: scratch of 4 V_l + nnz_l float4
// on levels >= 1, nnz_0 on level 0).
struct AdjLevel {
    float4 *coef = nullptr;   // V_l
    int *corner = nullptr;    // V_l
    int *pidx = nullptr;      // nnz_l, levels >= 1: the slot of each corner's contribution
    float *sh = nullptr;      // E_l, when adjoint_level_creased
};
bool adjoint_supported(const TopoImpl &T);
bool adjoint_level_creased(const TopoImpl &T, int l);
void adjoint_prepare(TopoImpl &T, int l, const AdjLevel &P, cudaStream_t s);
void adjoint_step(TopoImpl &T, int l, const float *G, bool G4, float *g, bool g4, const AdjLevel &P,
                  float4 *part, cudaStream_t s);
// alsub_mesh_create_ex behind the C ABI. B_stated null: the boundary edges are counted on the
// device and read back (the call synchronises `stream`); else the caller states their number and
// the count is checked on the device (mesh_boundary_check), so nothing waits for the device.
alsub_status create_mesh(alsub_scheme scheme, int32_t V, int32_t F, const int32_t *off_h, const int32_t *fv_h,
                         int32_t K, const int32_t *cv_h, const float *cs_h, const alsub_allocator *allocator,
                         const long long *B_stated, void *stream, alsub_mesh_t *out);

// The implementation behind a topology handle.
TopoImpl *topology_impl(alsub_topology_t h);
// Store the per-corner edge ids and twins of every level below the last one (the last
// Catmull-Clark step normally derives them on the fly); the operator builder reads them.
alsub_status ensure_helpers(TopoImpl &T, cudaStream_t s);

}  // namespace alsub
