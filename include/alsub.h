/*
 * alsub.h -- C ABI of libalsub, a GB300 (sm_103a) implementation of uniform subdivision as
 * sparse linear algebra on the oriented face-vertex mesh matrix (AlSub, Mlakar et al.,
 * arXiv 1809.06047).
 *
 * Scope: one uniform subdivision step, repeated level by level, for Catmull-Clark (Sec. 3),
 * Loop (Appendix B) and sqrt(3) (Appendix A) on 2-manifold meshes -- closed, or open with
 * boundaries for Catmull-Clark (Sec. 3.1 and 3.2 "Boundaries"), Loop and sqrt(3) (Kobbelt 2000) --
 * with sharp and semi-sharp creases for Catmull-Clark and Loop (Sec. 3.3) and infinitely sharp
 * ones for sqrt(3), and the extraction of selective subdivision
 * (Sec. 3.4). Topology refinement (the build step
 * of Fig. module_core) is integer work that emits each level's face table directly; vertex
 * refinement (the eval step) is FP32. The subdivision operator of Sec. 3.6 "Single SpMV
 * evaluation" (R_i per level, or the composite R = R_{L-1} ... R_0) can be built once and applied
 * as one SpMV per frame, and applied transposed for gradients; so can the composition of a chain of
 * selective refinement rounds (feature-adaptive subdivision).
 *
 * Conventions shared by every call:
 *  - Every call returns an alsub_status and never aborts, traps or exits. On failure
 *    alsub_last_error() returns a message for the calling thread.
 *  - Pointers named *_host are host memory and are only read during the call. Pointers named
 *    *_dev are device memory owned by the caller, on the current CUDA device, and must stay
 *    valid until the work enqueued on `stream` has completed.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *    enqueued on it without an implicit device synchronisation, except in the calls that say
 *    they synchronise.
 *  - Handles own the device memory they allocate; their destroy call frees it (stream ordered on
 *    the stream they were created with).
 *  - Errors found on the device (a non-manifold input, a valence beyond the supported bound)
 *    are latched in a per-handle device status word and reported by alsub_topology_status(),
 *    which synchronises the handle's stream.
 *  - Vertex positions are FP32 xyz, packed as float[3*V] (12 bytes per vertex, AoS).
 *  - Indices are int32; every per-level count of vertices, faces, corners and edges must stay
 *    below 2^31 - 1 (ALSUB_ERR_UNSUPPORTED otherwise).
 *
 * Vertex numbering of a refined level follows the paper's refined mesh matrix (Sec. 3.2,
 * "Topology refinement"): the old vertices keep their ids, then one face point per face
 * (Catmull-Clark, sqrt(3): id |v| + r), then one edge point per edge (Catmull-Clark:
 * |v| + |f| + e; Loop: |v| + e). Faces of level l+1 are the children of level l's faces in
 * corner order: Catmull-Clark corner x of face r gives quad x = [v_x, e(x), f_r, e(prev x)];
 * Loop triangle r gives 4r..4r+3 = [v0,e0,e2], [v1,e1,e0], [v2,e2,e1], [e0,e1,e2]; sqrt(3)
 * corner x of triangle r gives triangle x = [v_x, f_{F(next x, x)}, f_r]. Edge ids are free
 * (Sec. 3.2 only asks for a unique enumeration); this library numbers them level by level as
 * described under alsub_refine_topology below.
 */
#ifndef ALSUB_H
#define ALSUB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ALSUB_OK = 0,
    ALSUB_ERR_INVALID_ARG = 1,   /* a pointer, count, index or sharpness out of range */
    ALSUB_ERR_NONMANIFOLD = 2,   /* duplicate directed edge, edge of >2 faces, vertex with >1 fan */
    ALSUB_ERR_UNSUPPORTED = 3,   /* crease at a boundary, counts beyond int32, valence > 1024, a
                                    call with no path for the mesh */
    ALSUB_ERR_OOM = 4,           /* device allocation failed or a budget is exhausted */
    ALSUB_ERR_TIMEOUT = 5,       /* a bounded wait ran out */
    ALSUB_ERR_DEVICE = 6,        /* a CUDA runtime error */
    ALSUB_ERR_BUSY = 7,          /* the server has no free slot and the request was not queued */
    ALSUB_ERR_NOT_READY = 8      /* the request is still in flight */
} alsub_status;

typedef enum { ALSUB_CATMULL_CLARK = 0, ALSUB_LOOP = 1, ALSUB_SQRT3 = 2 } alsub_scheme;

typedef struct alsub_mesh_s *alsub_mesh_t;
typedef struct alsub_topology_s *alsub_topology_t;
typedef struct alsub_operator_s *alsub_operator_t;
typedef struct alsub_server_s *alsub_server_t;

/* Message of the last failed call on this thread ("" if none). Never NULL. */
const char *alsub_last_error(void);

/* Static name of a status code. */
const char *alsub_status_string(alsub_status s);

/*
 * Copy `bytes` bytes between host and/or device buffers (unified addressing decides the
 * direction) on `stream`, then synchronise that stream. Plumbing for bindings that hold raw
 * device pointers returned by the accessors below. Errors: INVALID_ARG, DEVICE.
 */
alsub_status alsub_copy(void *dst, const void *src, size_t bytes, void *stream);

/*
 * Closed-form per-level counts (host only, no GPU needed). Sec. 3.1 step 4 / Sec. 3.2 for
 * Catmull-Clark (V' = V + F + E, F' = nnz, nnz' = 4 nnz, E' = 2E + nnz), Appendix B for Loop
 * (V' = V + E, F' = 4F, E' = 2E + 3F), Appendix A for sqrt(3) (V' = V + F, F' = 3F,
 * E' = E + 3F); a closed mesh has E = nnz / 2.
 *   counts_host: int64[4 * (levels + 1)], filled with (V, F, nnz, E) per level.
 * Errors: INVALID_ARG for negative or inconsistent inputs, UNSUPPORTED when a count would exceed
 * int32 or nnz is odd (an open mesh: see alsub_plan_open).
 */
alsub_status alsub_plan(alsub_scheme scheme, int64_t num_verts, int64_t num_faces, int64_t nnz,
                        int32_t levels, int64_t *counts_host);

/*
 * alsub_plan for a mesh with `boundary_edges` edges of one face (Sec. 3.1 and 3.2 "Boundaries"):
 * E = (nnz + boundary_edges) / 2 on level 0, the same recurrences after it, each boundary edge
 * splitting into two (Catmull-Clark, Loop). sqrt(3) (Kobbelt 2000) alternates two kinds of step:
 * from an even level the boundary edges stay (the recurrences above); from an odd level each splits
 * into three, which adds one vertex and one edge per boundary edge (V' = V + F + B, E' = E + 3F +
 * B, B' = 3B). boundary_edges = 0 is alsub_plan.
 * Errors: those of alsub_plan; INVALID_ARG when nnz + boundary_edges is odd or boundary_edges is
 * negative or above nnz.
 */
alsub_status alsub_plan_open(alsub_scheme scheme, int64_t num_verts, int64_t num_faces, int64_t nnz,
                             int64_t boundary_edges, int32_t levels, int64_t *counts_host);

/*
 * Create a control mesh: the reduced mesh matrix M of Sec. 4.1 as a face table, plus the crease
 * matrix C of Sec. 3.3 as a list of tagged edges.
 *   face_offsets_host: int32[num_faces + 1] CSR offsets, or NULL when every face has the
 *                      scheme's order (4 for a uniform Catmull-Clark quad mesh, 3 for Loop and
 *                      sqrt(3)).
 *   face_verts_host:   int32[nnz] vertex ids of each face in counter-clockwise cyclic order.
 *   crease_verts_host: int32[2 * num_creases] edge endpoints; crease_sharpness_host: float[K]
 *                      sharpness sigma >= 0 (+inf = infinitely sharp; 0 = smooth, dropped).
 *                      sqrt(3) (no crease rules in the paper) keeps the infinitely sharp creases
 *                      as feature edges, like its boundary edges below; finite sharpness is
 *                      ignored.
 * The host validates ranges (vertex ids, face order >= 3, Loop/sqrt(3) triangles only, no
 * repeated vertex in a face, every vertex used, sigma not NaN or negative) and copies everything
 * to the device on `stream`; the caller may free its arrays on return. Adjacency is checked on
 * the device when a topology is built.
 * Catmull-Clark meshes may be open (Sec. 3.1 and 3.2 "Boundaries"): an edge of one face is a
 * boundary edge, refined by the midpoint rule, and a vertex on boundary edges by Eq. CC_boundary
 * (3/4 p + 1/8 of its two boundary neighbours). The create call counts the boundary edges on the
 * device (it synchronises `stream`); alsub_mesh_boundary_edges reports the count, which sizes the
 * levels (alsub_plan_open). A vertex must lie on at most two boundary edges (one fan; checked when
 * the topology is built), and no crease may touch a boundary vertex (the paper defines no such
 * combination: UNSUPPORTED). Loop meshes may be open too, with the same two boundary rules (Appendix
 * B gives Loop none of its own; these keep its boundary the cubic B-spline curve of the control
 * polygon, as for Catmull-Clark). sqrt(3) meshes may be open too (Appendix A omits boundaries; the
 * treatment is Kobbelt 2000's): boundary edges and infinitely sharp creases (feature edges) are not
 * flipped on the first step of each pair of steps and are split into three on the second, their
 * curves refined by the ternary cubic B-spline rules (new points (1, 16, 10) / 27 and
 * (10, 16, 1) / 27, curve vertices (4, 19, 4) / 27 on the second step and unmoved on the first,
 * corners fixed, a curve end mirrored). Such meshes take a general per-level path (every level's
 * twins stored); the operator and ragged batches refuse them (UNSUPPORTED).
 * Errors: INVALID_ARG, NONMANIFOLD (a repeated directed edge found by the boundary count),
 * UNSUPPORTED (counts beyond int32, a crease at the boundary), OOM, DEVICE.
 */
alsub_status alsub_mesh_create(alsub_scheme scheme, int32_t num_verts, int32_t num_faces,
                               const int32_t *face_offsets_host, const int32_t *face_verts_host,
                               int32_t num_creases, const int32_t *crease_verts_host,
                               const float *crease_sharpness_host, void *stream,
                               alsub_mesh_t *out);

/*
 * Device memory supplied by the caller (the boundary's allocator callback: a caller that manages
 * device memory itself, e.g. through PyTorch's caching allocator or a fixed arena, keeps every
 * array of the library inside it). alloc returns `bytes` of device memory usable in stream order
 * on `stream` (16-byte aligned; a misaligned block is handed back and the call fails with OOM),
 * or NULL when it has none (the library call then fails with OOM); free takes back a block once
 * the work that the library enqueued on `stream` before the call no longer needs it (stream
 * ordered, like cudaFreeAsync). ctx is passed through. Both callbacks must be thread-safe if the
 * caller uses the library from several threads, and must not call back into the library.
 */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx, void *stream);
    void (*free)(void *ptr, void *ctx, void *stream);
    void *ctx;
} alsub_allocator;

/*
 * alsub_mesh_create with the caller's allocator (NULL: CUDA's stream-ordered allocator, as
 * alsub_mesh_create). The mesh and every handle made from it (topologies and their host-buffer
 * staging, operators, hierarchical edits, extracted and reordered meshes, which inherit the
 * allocator) take all of their device memory, temporaries included, from `allocator`; the
 * allocator struct is copied, and its callbacks and ctx must stay valid until the last of those
 * handles is destroyed. Batches and servers keep using their own allocations. Errors: those of
 * alsub_mesh_create, INVALID_ARG when alloc or free is NULL.
 */
alsub_status alsub_mesh_create_ex(alsub_scheme scheme, int32_t num_verts, int32_t num_faces,
                                  const int32_t *face_offsets_host, const int32_t *face_verts_host,
                                  int32_t num_creases, const int32_t *crease_verts_host,
                                  const float *crease_sharpness_host, const alsub_allocator *allocator,
                                  void *stream, alsub_mesh_t *out);

alsub_status alsub_mesh_destroy(alsub_mesh_t mesh);

/* Number of boundary edges (edges of one face) of a mesh; 0 for a closed mesh. Host only.
 * Errors: INVALID_ARG. */
alsub_status alsub_mesh_boundary_edges(alsub_mesh_t mesh, int64_t *boundary_edges);

/* Scheme, vertex, face, corner and crease counts of a mesh (host only; any pointer may be NULL).
 * Errors: INVALID_ARG. */
alsub_status alsub_mesh_info(alsub_mesh_t mesh, int32_t *scheme, int64_t *num_verts, int64_t *num_faces,
                             int64_t *nnz, int64_t *num_creases);

/*
 * Selective subdivision (Sec. 3.4, Fig. module_selective): extract the region around selected
 * vertices of level `level` (0 = the control mesh) of a built Catmull-Clark or Loop topology as a
 * new mesh,
 * which the ordinary calls then refine (it is open: its cut is refined by the boundary rules, so
 * only faces about two rings inside it match the uniform refinement).
 *   select_dev: uint8[V_level] on the device, 1 = selected; NULL selects the extraordinary vertices
 *               (valence != 4 for Catmull-Clark, != 6 for Loop, Eq. vo, among the vertices on no
 *               boundary edge) and both ends of every live crease of the level.
 *   rings >= 1: propagation steps q = M^T x (faces with a selected vertex), x = M q (their vertices);
 *               the mesh keeps the faces of the last q and their vertices, in their original order
 *               (M' = X M X-ring with X, X-ring rows / columns of the identity), and the creases
 *               whose both ends have every face around them kept.
 * The new handle owns its arrays and the maps (alsub_mesh_extract_maps); positions follow with
 * alsub_mesh_gather. Synchronises `stream` (the sizes are read back). Errors: INVALID_ARG (bad
 * level or rings, topology not built, nothing selected), UNSUPPORTED (sqrt(3): the extracted mesh is
 * open), OOM, DEVICE.
 */
alsub_status alsub_topology_extract(alsub_topology_t topo, int32_t level, const uint8_t *select_dev,
                                    int32_t rings, void *stream, alsub_mesh_t *out);

/*
 * Regular-patch evaluation (Sec. 3.4, the other half of feature-adaptive subdivision: faces whose
 * vertices all have valence 4 are bicubic B-spline patches whose limit surface is evaluated
 * directly). A face of level `level` (0 .. levels - 1 of a built Catmull-Clark topology: the level
 * needs its twins) is regular when its 3 x 3 block of faces is 9 quads around its 4 interior
 * valence-4 vertices and no live crease touches the block's 16 vertices.
 * alsub_topology_regular_faces: flags_dev uint8[F_level] = 1 for the regular faces; *count (when
 *   not NULL) receives their number, which synchronises `stream`.
 * alsub_topology_eval_patches: for face faces_dev[i] (int32[n]) samples the patch at the
 *   samples x samples grid u = a / (samples - 1), v = b / (samples - 1) (u along the face's corner
 *   0 -> 1, v along corner 0 -> 3; samples = 1 gives u = v = 0) from the level's positions P_dev
 *   (float[3 V_level], packed xyz) into out_dev float[3 * n * samples^2] (patch i, row b, column a);
 *   a face that is not regular gets NaN. Uniform cubic B-spline basis, FP32.
 * Errors: INVALID_ARG (level, sizes, NULL), UNSUPPORTED (Loop, sqrt(3)), OOM, DEVICE.
 */
alsub_status alsub_topology_regular_faces(alsub_topology_t topo, int32_t level, uint8_t *flags_dev, int64_t *count,
                                          void *stream);
alsub_status alsub_topology_eval_patches(alsub_topology_t topo, int32_t level, int32_t n, const int32_t *faces_dev,
                                         const float *P_dev, int32_t samples, float *out_dev, void *stream);

/*
 * Mesh reordering (Sec. 4.5): a new mesh with the same faces, vertices renumbered by reverse
 * Cuthill-McKee (Cuthill and McKee 1969, reversed as in George 1971) on the graph of the mesh
 * Laplacian (u ~ w when an edge of some face joins them) and faces sorted by their first non-zero
 * row of M, i.e. by the least new index among their vertices.
 *   Cuthill-McKee: each connected component starts at its unlabelled vertex of least (degree,
 *   index); labelled vertices are visited in label order and each labels its unlabelled neighbours
 *   in increasing (degree, index); the new index of a vertex is V - 1 - its label. Faces with the
 *   same least vertex keep their input order; each face keeps its corners in order from the same
 *   first corner; creases keep their order with their ends renamed. The result is unique.
 * Runs on the device, one breadth-first level at a time (synchronises `stream` once per level).
 * The new handle owns its arrays and the maps (alsub_mesh_extract_maps: vmap[new] = old vertex,
 * fmap[new] = old face); positions follow with alsub_mesh_gather. *levels (may be NULL): the
 * breadth-first levels it took. Errors: INVALID_ARG (NULL), UNSUPPORTED (more than 2^30 corners),
 * OOM, DEVICE.
 */
alsub_status alsub_mesh_reorder(alsub_mesh_t mesh, void *stream, alsub_mesh_t *out, int32_t *levels);

/* Device arrays of a mesh (owned by it; any pointer may be NULL): off int32[F + 1], fv int32[nnz],
 * crease ends int32[2K] and sharpness float[K] (NULL when K = 0; creases of sharpness 0 were
 * dropped at creation). Read them after the call that made the mesh has completed on its stream.
 * Errors: INVALID_ARG. */
alsub_status alsub_mesh_arrays(alsub_mesh_t mesh, const int32_t **off_dev, const int32_t **fv_dev,
                               const int32_t **crease_verts_dev, const float **crease_sharp_dev);

/* Device maps of an extracted or reordered mesh (owned by it): vmap[i] = the source vertex of
 * vertex i (int32[V']), fmap[f] = the source face of face f (int32[F']). Errors: INVALID_ARG (a
 * mesh made by alsub_mesh_create has no maps). */
alsub_status alsub_mesh_extract_maps(alsub_mesh_t mesh, const int32_t **vmap_dev, const int32_t **fmap_dev);

/* P' = X P for an extracted or reordered mesh: row i of out_dev (float[3 V']) = row vmap[i] of P_dev
 * (the source's positions, float[3 V_source]); enqueued on `stream`. Errors: INVALID_ARG, DEVICE. */
alsub_status alsub_mesh_gather(alsub_mesh_t mesh, const float *P_dev, float *out_dev, void *stream);

/*
 * Build the topology of `levels` uniform refinement steps (the build step of Fig. module_core,
 * Sec. 3.6 "Static topology"): for every level the face table M_{l+1}, the per-corner edge
 * numbering (E, Eq. CC_E; Appendix B for Loop) and the per-corner face adjacency (F, Eq. F), and
 * the inherited crease lists (Sec. 3.3). Level 0 edges are numbered by an exclusive scan over
 * the corners that own their edge (a -> b with a < b, or a boundary corner: no twin, twin -1 in
 * the per-corner adjacency of every level); each refined level numbers the two halves
 * of parent edge e as 2e and 2e+1 and the edges interior to parent faces after them. All sizes
 * are closed-form, so nothing is read back to the host. The handle keeps every level resident
 * for alsub_refine_vertices and alsub_build_operator. Enqueued on `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, DEVICE; adjacency errors are latched on the device
 * (see alsub_topology_status).
 */
alsub_status alsub_refine_topology(alsub_mesh_t mesh, int32_t levels, void *stream,
                                   alsub_topology_t *out);

/*
 * Allocate a topology handle for `levels` steps of `mesh` without computing anything (sizes are
 * closed-form). alsub_subdivide fills it; alsub_refine_topology is alsub_topology_create plus the
 * build. The handle keeps a reference to `mesh`, which must outlive every call on it but
 * alsub_topology_destroy (the release reads nothing of the mesh: the two may be destroyed in
 * either order).
 * Errors: INVALID_ARG, UNSUPPORTED (a level beyond int32 counts), OOM, DEVICE.
 */
alsub_status alsub_topology_create(alsub_mesh_t mesh, int32_t levels, void *stream,
                                   alsub_topology_t *out);

/* Synchronise the handle's stream and return its latched device status (OK, NONMANIFOLD,
 * UNSUPPORTED or INVALID_ARG for a crease that is not an edge). */
alsub_status alsub_topology_status(alsub_topology_t topo);

/*
 * Sizes and device face table of one level (0 <= level <= levels).
 *   face_verts_dev: level 0: the input face table (face_offsets_dev gives its CSR offsets);
 *                   level >= 1: int32[nnz], 4 per face for Catmull-Clark, 3 for Loop/sqrt(3)
 *                   (face_offsets_dev is then NULL). Owned by the handle.
 * Any out pointer may be NULL.
 */
alsub_status alsub_topology_level(alsub_topology_t topo, int32_t level, int64_t *V, int64_t *F,
                                  int64_t *nnz, int64_t *E, const int32_t **face_offsets_dev,
                                  const int32_t **face_verts_dev);

/*
 * Crease list of one level (Sec. 3.3: the crease matrix C_l as tagged edges). Synchronises the
 * handle's stream to read the count. crease_verts_dev: int32[2K] endpoints, crease_sharp_dev:
 * float[K]; both owned by the handle. Inherited sharpness is computed in FP32 in the fixed order
 * t = 3 sigma; u = sigma_o + t; w = 0.25 u; y = w - 1; max(y, 0), where sigma_o is the other
 * crease at the end vertex when exactly two creases meet there and it is finite, else sigma.
 */
alsub_status alsub_topology_creases(alsub_topology_t topo, int32_t level, int32_t *K,
                                    const int32_t **crease_verts_dev,
                                    const float **crease_sharp_dev);

alsub_status alsub_topology_destroy(alsub_topology_t topo);

/*
 * Vertex refinement of all levels of a built topology (the eval step: Sec. 3.2 face, edge and
 * vertex points as mapped SpMVs, fused in one pass per level; crease rules overwrite crease
 * vertices and edge points, Fig. module_creases).
 *   P0_dev: float[3 * V_0]; PL_dev: float[3 * V_levels].
 *   scratch_dev: NULL (use the handle's own buffers; then calls on one handle must not overlap)
 *                or device memory of alsub_refine_vertices_scratch_bytes() bytes.
 * Crease rules: edge point sigma >= 1 -> midpoint, 0 < sigma < 1 -> (1 - sigma) smooth + sigma
 * midpoint; vertex with k incident creases, mean sharpness s: k < 2 smooth, k == 2
 * (p_a + 6 p + p_b) / 8, k >= 3 p, blended w sharp + (1 - w) smooth with w = min(s, 1).
 */
alsub_status alsub_refine_vertices(alsub_topology_t topo, const float *P0_dev, float *PL_dev,
                                   void *scratch_dev, void *stream);
alsub_status alsub_refine_vertices_scratch_bytes(alsub_topology_t topo, size_t *bytes);

/*
 * Dynamic-topology subdivision (Sec. 3.6 "Dynamic topology"): rebuild the whole topology of the
 * handle from its control mesh AND refine the vertices, one fused build+eval pass per level, so
 * a topology-changing edit costs one call with no preprocessing. The per-corner adjacency of the
 * last level is not stored (nothing consumes it); face tables and crease lists of every level
 * are. Same arguments as alsub_refine_vertices.
 */
alsub_status alsub_subdivide(alsub_topology_t topo, const float *P0_dev, float *PL_dev,
                             void *scratch_dev, void *stream);

/*
 * alsub_subdivide with the control positions and the result in HOST memory: the call copies
 * P0_host (float[3 * V_0]) into page-locked staging before it returns (the caller may reuse the
 * buffer at once), uploads it, runs the dynamic-topology subdivision into one of two device
 * buffers the handle owns, and downloads the result into PL_host (float[3 * V_levels];
 * page-locked memory is written by DMA, pageable memory through the runtime's staging). `stream`
 * completes when PL_host holds the result, so synchronising it (or an event recorded on it)
 * publishes the result. The upload and eval run on a private stream and the download on another:
 * call k + 1's upload and eval overlap call k's download (double-buffered on the device), so a
 * sequence of calls moves at the pace of the slower of the two. A caller must not read PL_host of
 * call k while a later call that writes the same buffer may be in flight. The handle's device
 * buffers (2 x 12 V_levels bytes plus 12 V_0) are allocated at the first call and freed with the
 * handle. Errors: INVALID_ARG, OOM, DEVICE and those of alsub_subdivide.
 */
alsub_status alsub_subdivide_host(alsub_topology_t topo, const float *P0_host, float *PL_host, void *stream);

/*
 * Hierarchical edits / displacement between levels (Sec. 3.5 "Other effects": the vertex data of
 * every level is at hand after its iteration and may be modified before the next one). After level
 * `level` (1 .. levels) has been refined (smooth rules, crease fix, boundary repair), offset i
 * (off_dev[3i .. 3i+2]) is added to vertex vid_dev[i] of that level, before the next step reads it
 * or, for the last level, in the output. The ids of one level must be distinct; an id out of range
 * latches INVALID_ARG. The arrays are copied (device or host memory); n = 0 clears the level's
 * edits. Applied by alsub_refine_vertices, alsub_subdivide and alsub_subdivide_host; operators
 * ignore them (with edits the result is R P_0 plus the refined edits, no longer R P_0).
 * Synchronises the handle's and `stream`'s work (calls in flight may read the old edits).
 * Errors: INVALID_ARG, OOM, DEVICE.
 */
alsub_status alsub_topology_set_edits(alsub_topology_t topo, int32_t level, int32_t n, const int32_t *vid_dev,
                                      const float *off_dev, void *stream);

/*
 * Subdivision operator (Sec. 3.6 "Single SpMV evaluation", Eq. singleSpMV): R_l maps the positions
 * of level l to those of level l+1 (P_{l+1} = R_l P_l), R = R_{L-1} ... R_0 maps the control mesh
 * to the last level. Built from a built topology in the paper's two stages (count the non-zeros
 * of every row, then fill column indices and FP32 weights); rows are sorted by column.
 *   flags: ALSUB_OP_CHAIN keeps every R_l (apply = L SpMVs); ALSUB_OP_COMPOSE forms R by row-wise
 *          sparse products (apply = one SpMV; memory ~ rows x support); ALSUB_OP_TRANSPOSE also
 *          builds the transposes for alsub_apply_operator_transpose (the adjoint g_0 = R^T g_L);
 *          ALSUB_OP_MATRIX_FREE applies R without storing it: its rows are the stencils the eval
 *          kernels evaluate from the cached topology (apply = alsub_refine_vertices' kernels, in
 *          the operator's own scratch, a repeated apply replaying a captured graph), which moves the
 *          face tables of the levels and their positions instead of ~16 column indices and weights
 *          per refined vertex. Its transpose, on a closed Catmull-Clark mesh, is matrix-free too:
 *          g_l = R_l^T g_{l+1} gathered per coarse vertex (its face points, the edge points around
 *          and across its faces, its own and its neighbours' vertex points, with the crease rules),
 *          no atomics, in two passes per level (per coarse face its contribution at each corner,
 *          then per coarse vertex the sum of its contributions), from per-vertex coefficients and
 *          per-corner slots computed once here (about 40 bytes per vertex of every level below the
 *          last, and the levels' edge ids and twins, which are then stored), with a scratch of
 *          16 bytes per contribution of the largest such level (about 128 bytes per vertex) and
 *          two levels of gradients. With
 *          ALSUB_OP_TRANSPOSE (and no other flag) the transposes of the R_l are stored and applied
 *          instead (any scheme). When combined with CHAIN or COMPOSE, apply takes the matrix-free
 *          form and alsub_operator_info the stored matrices.
 * Weights: Catmull-Clark face row 1/c; edge row 1/4 on the endpoints and 1/(4c) on every vertex of
 * both faces (Eq. 2 with Eq. 1 expanded); vertex row (1 - 2/n) on the vertex, 1/n^2 on each
 * neighbour and 1/(n^2 c) on every vertex of each incident face (Eq. pos_update); Loop and sqrt(3)
 * per Appendices B and A; crease rows blended as in alsub_refine_vertices.
 * The operator keeps a pointer to the topology, which must outlive every call on it but
 * alsub_operator_destroy (which reads nothing of the topology). Synchronises `stream`
 * (the non-zero counts size the allocations).
 * Errors: INVALID_ARG (topology not built, no flags), UNSUPPORTED (a stencil row of more than 192
 * entries; a sqrt(3) mesh with boundaries or infinitely sharp creases), OOM, DEVICE.
 */
typedef enum {
    ALSUB_OP_CHAIN = 1,
    ALSUB_OP_COMPOSE = 2,
    ALSUB_OP_TRANSPOSE = 4,
    ALSUB_OP_MATRIX_FREE = 8,
    ALSUB_OP_STACKED = 16          /* alsub_build_adaptive_operator only */
} alsub_operator_flags;

alsub_status alsub_build_operator(alsub_topology_t topo, uint32_t flags, void *stream,
                                  alsub_operator_t *out);

/*
 * Size and device CSR arrays of one matrix of the operator: level >= 0 for R_level (needs
 * ALSUB_OP_CHAIN), level < 0 for the composite R (needs ALSUB_OP_COMPOSE). rowptr: int64[rows+1],
 * col: int32[nnz], w: float[nnz], owned by the operator. Any out pointer may be NULL.
 */
alsub_status alsub_operator_info(alsub_operator_t op, int32_t level, int64_t *rows, int64_t *cols,
                                 int64_t *nnz, const int64_t **rowptr_dev, const int32_t **col_dev,
                                 const float **w_dev);

/* P_L = R P_0 on `stream` (matrix-free: the eval kernels; else one SpMV with the composite, else
 * the chain of R_l). P0_dev: float[3 V_0], PL_dev: float[3 V_L] (packed xyz). A matrix-free
 * operator keeps its intermediate levels in its own scratch: its applies are taken one at a time
 * on the host and ordered on the device (each waits on the stream for the previous one), and the
 * result is bitwise that of alsub_refine_vertices on the same topology. Calls on one chain
 * operator must not overlap (it keeps intermediate levels in the operator). */
alsub_status alsub_apply_operator(alsub_operator_t op, const float *P0_dev, float *PL_dev, void *stream);

/* g_0 = R^T g_L (the adjoint of vertex refinement: vertex refinement is linear in P, so this is
 * the exact gradient of any loss of P_L with respect to P_0 given g_L = dLoss/dP_L). Needs
 * ALSUB_OP_TRANSPOSE (the stored transposes), or ALSUB_OP_MATRIX_FREE on a closed Catmull-Clark
 * mesh (the per-vertex gather; its applies, like the forward ones, run one at a time and in
 * order on the device). gL_dev: float[3 V_L], g0_dev: float[3 V_0]. Errors: INVALID_ARG when the
 * operator has neither. */
alsub_status alsub_apply_operator_transpose(alsub_operator_t op, const float *gL_dev, float *g0_dev,
                                            void *stream);

/*
 * Feature-adaptive single-SpMV operator (Sec. 3.4, Fig. module_selective, evaluated as Sec. 3.6
 * "Single SpMV evaluation" and Sec. 5 "Adaptive Subdivision" do): after the build, one SpMV takes
 * the control points to every refined point of a chain of selective refinement rounds,
 *   R = R^(n-1) X^(n-1) ... R^(1) X^(1) R^(0),
 * where R^(k) = R_{L_k - 1} ... R_0 composes the levels of topos[k] (the identity when it has none)
 * and X^(k) is the extraction matrix of topos[k]'s mesh: row i is e_{vmap[i]} over the vertices of
 * the level it was extracted from. topos[0] is any built topology of the control mesh; for k >= 1
 * topos[k] must be built on a mesh that alsub_topology_extract took from the last level of
 * topos[k - 1] (checked from the handles; INVALID_ARG otherwise). All n topologies are read during
 * the build only: the operator keeps nothing of them, and they may be destroyed afterwards.
 *   flags: ALSUB_OP_TRANSPOSE also stores R^T (alsub_apply_operator_transpose);
 *          ALSUB_OP_STACKED stacks the rounds: rows are the last level of topos[0], then that of
 *          topos[1], ... (the points every round's patches and faces need), instead of the last
 *          round's only. Other flags are INVALID_ARG.
 * alsub_operator_info(op, -1, ...) gives the matrix (rows = the output points, cols = V of topos[0]'s
 * control mesh); alsub_apply_operator computes P_out = R P_0 with P0_dev float[3 cols] and PL_dev
 * float[3 rows]. Synchronises `stream` (the non-zero counts size the allocations) and each
 * topology's stream (a topology whose device status latched an error fails the build with it).
 * Errors: INVALID_ARG (NULL, n < 1, a topology not built, a chain that is not one), UNSUPPORTED (a
 * stencil row of more than 192 entries; a sqrt(3) mesh with boundaries or infinitely sharp
 * creases), OOM, DEVICE.
 */
alsub_status alsub_build_adaptive_operator(const alsub_topology_t *topos, int32_t n, uint32_t flags,
                                           void *stream, alsub_operator_t *out);

alsub_status alsub_operator_destroy(alsub_operator_t op);

/*
 * Ragged batches (no counterpart in the paper's text; it processes one mesh per call): vertex
 * refinement of n built topologies of uneven sizes, any mix of schemes and level counts, with one
 * kernel launch per level per kernel class over a flattened work list of face tiles (per-member
 * closed-form sizes; persistent grid). Member i reads P0_dev[i] (float[3 V_0]) and writes PL_dev[i]
 * (float[3 V_L]) exactly as alsub_refine_vertices(topos[i], ...) would, using that topology's own
 * scratch, so a topology may appear only once and must not be refined elsewhere while the batch
 * runs. The buffers are bound at creation: to refine new positions, write them into P0_dev[i].
 * Members must be closed meshes without sqrt(3) feature edges (UNSUPPORTED otherwise: the batch
 * has no boundary repair step and does not run the sqrt(3) feature path).
 * Members' hierarchical edits (alsub_topology_set_edits) are applied as set when the batch first
 * runs on a stream (its captured graph keeps them).
 */
typedef struct alsub_batch_s *alsub_batch_t;

alsub_status alsub_batch_create(int32_t n, const alsub_topology_t *topos, const float *const *P0_dev,
                                float *const *PL_dev, alsub_batch_t *out);

/* Run the batch on `stream`. On a non-default stream the first call captures the whole launch
 * sequence into a CUDA graph, later calls on that stream replay it. */
alsub_status alsub_batch_refine(alsub_batch_t batch, void *stream);

/* Set the block size (128, 256 or 512 faces per tile) and the persistent grid (blocks per SM,
 * 0 = one block per tile); synchronises the device. */
alsub_status alsub_batch_configure(alsub_batch_t batch, int32_t block, int32_t blocks_per_sm);

/* Autotuner: time every block size x persistence candidate on this batch (2 warm-up and 5 timed
 * runs each, CUDA events on `stream`), keep the fastest and return it. */
alsub_status alsub_batch_tune(alsub_batch_t batch, void *stream, int32_t *block,
                              int32_t *blocks_per_sm, float *best_ms);

/* Kernels launched by all alsub_batch_refine calls so far. */
alsub_status alsub_batch_launches(alsub_batch_t batch, int64_t *launches);

alsub_status alsub_batch_destroy(alsub_batch_t batch);

/*
 * Live timing of the library's own work on the calling stream. capacity > 0 allocates
 * capacity x (levels + 2) CUDA events and makes every following alsub_subdivide /
 * alsub_refine_vertices call on the handle record one event before its level-0 build, one after
 * it, and one after each level's kernels; capacity = 0 turns timing off. Calls beyond `capacity`
 * since the last read make the read fail with INVALID_ARG. Errors: INVALID_ARG, OOM, DEVICE.
 */
alsub_status alsub_topology_set_timing(alsub_topology_t topo, int32_t capacity);

/*
 * Read and reset the timings (synchronises the handle's stream).
 *   ms_host: double[levels + 1]: [0] summed duration of the level-0 builds, [1 + l] summed
 *            duration of level l's step (the l -> l+1 build and/or eval kernels, crease kernels
 *            included), over the `*calls` calls recorded since the last read.
 *   launches: number of kernels the handle launched since the last read (all calls, timed or not).
 */
alsub_status alsub_topology_timings(alsub_topology_t topo, double *ms_host, int32_t *calls,
                                    int64_t *launches);

/*
 * Vertex refinement that allocates nothing. The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory at the point where they refine (for example
 * code running inside another allocator's callback, or a process that forbids device allocation
 * after start-up) and cannot pass a scratch buffer of their own.
 * It computes exactly what alsub_refine_vertices computes, with the intermediate levels held in a
 * fixed 32 MiB array compiled into the library instead of the handle's or the caller's scratch,
 * and with its kernels launched directly on `stream`: it never captures or replays a CUDA graph
 * and makes no stream or event, so after its set-up it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   P0_dev: float[3 * V_0]; PL_dev: float[3 * V_levels]; both caller-owned device memory on the
 *   current device, which must also be the device the topology was created on.
 * Set-up: the first call on a device looks up the array's device address with that device
 * current. That lookup loads the part of the library that holds the array, which reserves its
 * 32 MiB on the device until the process exits (OOM if it cannot), and the first launch of each
 * kernel may load that kernel's code. So make the first call at start-up, before any stream
 * capture and before the point where allocation is forbidden. All calls share the one array and
 * it keeps the last call's contents (nothing in it needs to start at zero): calls that overlap on
 * the GPU race, so serialise them (one stream, or events).
 * Errors: INVALID_ARG (NULL argument, topology not built, topology on another device),
 * UNSUPPORTED when the topology's intermediate levels need more than 32 MiB
 * (alsub_refine_vertices_scratch_bytes tells the need), OOM (set-up), DEVICE.
 */
alsub_status alsub_refine_vertices_static(alsub_topology_t topo, const float *P0_dev, float *PL_dev,
                                          void *stream);

/*
 * Device bytes that alsub_topology_create(levels) allocates for a mesh of these sizes (host only,
 * no GPU needed; the same closed-form sizes the create call uses). boundary_edges as in
 * alsub_plan_open (0 for a closed mesh). sigma_max is the largest crease sharpness (+inf
 * allowed; it bounds how many levels keep crease lists). For sqrt(3), num_creases counts the
 * infinitely sharp creases (the only ones it keeps) and matters only when sigma_max is +inf. The
 * mesh itself holds 4 (F + 1) + 4 nnz + 12 K bytes more. Errors: those of alsub_plan_open.
 */
alsub_status alsub_plan_bytes(alsub_scheme scheme, int32_t num_verts, int32_t num_faces, int32_t nnz,
                              int32_t boundary_edges, int32_t num_creases, float sigma_max, int32_t levels,
                              size_t *bytes);

/* Device bytes a handle holds now (grows when alsub_build_operator stores the per-corner arrays
 * of a level that did not keep them). */
alsub_status alsub_topology_bytes(alsub_topology_t topo, size_t *bytes);
alsub_status alsub_operator_bytes(alsub_operator_t op, size_t *bytes);

/*
 * Serving loop (no counterpart in the paper's text; its "Static topology" mode of Sec. 3.6, build
 * once and evaluate every frame, is what the resident cache serves). A worker thread owned by the
 * server admits queued requests first come first served into `max_slots` slots, each with its own
 * CUDA stream, as soon as a slot is free and the request's device bytes fit the HBM budget, so
 * requests overlap on the GPU (continuous batching: a request joins as soon as another leaves).
 * Requests are one of:
 *   ALSUB_REQ_FRAME  new control positions for a resident topology (alsub_serve_register): one
 *                    SpMV with the cached composite operator, or the eval kernels on the cached
 *                    topology, as chosen when the resident was registered;
 *   ALSUB_REQ_MESH   a new control mesh: topology build and vertex refinement of every level in
 *                    one fused pass per level (alsub_subdivide), handles freed afterwards.
 * Admission counts, per request, the closed-form bytes of its topology (alsub_plan_bytes), its mesh
 * and its input/output positions (plus eval scratch for frames without an operator); residents
 * count their topology and operator for as long as the server lives. A request larger than the
 * budget left by the residents is refused at submit with ALSUB_ERR_OOM; if one is found over budget
 * at admission with nothing in flight it finishes with status ALSUB_ERR_OOM.
 * Latency of a request = completion seen by the worker (the slot's event done and the result in
 * host memory) - submit time; alsub_serve_stats gives percentiles over all completed requests.
 * While it lives the server raises the release threshold of the current device's default memory
 * pool to the budget (restored by alsub_serve_destroy), so stream-ordered allocations of
 * consecutive requests reuse memory instead of mapping it anew.
 */
typedef enum { ALSUB_REQ_FRAME = 0, ALSUB_REQ_MESH = 1 } alsub_request_kind;

typedef struct {
    int32_t kind;                          /* alsub_request_kind */
    int32_t resident;                      /* FRAME: id returned by alsub_serve_register */
    int32_t scheme;                        /* MESH: alsub_scheme */
    int32_t levels;                        /* MESH: refinement steps (0..15) */
    int32_t num_verts, num_faces;          /* MESH: as alsub_mesh_create */
    const int32_t *face_offsets_host;      /* MESH: as alsub_mesh_create (may be NULL) */
    const int32_t *face_verts_host;        /* MESH */
    int32_t num_creases;                   /* MESH */
    int32_t num_boundary_edges;            /* MESH: edges of one face (alsub_mesh_boundary_edges;
                                              0 for a closed mesh). It sizes V_L as
                                              alsub_plan_open does; a mesh with another count
                                              fails with INVALID_ARG. */
    const int32_t *crease_verts_host;      /* MESH */
    const float *crease_sharpness_host;    /* MESH */
    const float *P0_host;                  /* float[3 V_0]; copied by the submit call */
    float *PL_host;                        /* optional caller-owned output float[3 V_L], written
                                              before the request completes; page-locked memory is
                                              written by DMA, pageable memory through a staging
                                              copy. NULL: the server keeps the result until
                                              alsub_serve_release. */
} alsub_request;

typedef struct {
    int32_t status;                        /* the request's own outcome (alsub_status) */
    int32_t kind;
    int64_t num_verts;                     /* V_L */
    const float *PL_host;                  /* float[3 V_L]: the caller's buffer or the server's */
    double submit_s, start_s, done_s;      /* steady-clock seconds */
} alsub_result;

typedef struct {
    int64_t completed, failed, queued, in_flight;
    double p50_ms, p99_ms, mean_ms, max_ms;
    double throughput_rps;                 /* completed / (last completion - first submit) */
    uint64_t hbm_budget, hbm_in_use, hbm_peak;   /* admission accounting, bytes */
    int64_t frames_operator;               /* frames served by the cached composite operator */
    int64_t frames_eval;                   /* frames served by eval kernels on a cached topology */
    int64_t meshes;                        /* MESH requests completed */
    double host_start_ms_mean;             /* worker time to enqueue a request (validation,
                                              allocation, launches), mean over completed ones */
    double host_finish_ms_mean;            /* worker time to retire one (status, copies, frees) */
    int64_t peak_in_flight;                /* most requests admitted into slots and not yet
                                              retired at one time */
    int64_t device_overlap_peak;           /* most completed requests whose compute intervals on
                                              the device (CUDA events recorded on each request's
                                              stream after its input copy and after its kernels)
                                              were open at one instant: > 1 means the work of
                                              different requests overlapped on the GPU */
    double host_start_frame_ms_mean;       /* host_start_ms_mean over the FRAME requests */
    double host_start_mesh_ms_mean;        /* host_start_ms_mean over the MESH requests */
} alsub_serve_stats;

/* Start a server on the current device. max_slots 1..64 (concurrent requests), budget > 0. The
 * slots are served by max_slots / 2 worker threads (at most 8; the environment variable
 * ALSUB_SERVE_WORKERS sets another count, 1 .. max_slots).
 * Errors: INVALID_ARG, OOM, DEVICE. */
alsub_status alsub_serve_create(size_t hbm_budget_bytes, int32_t max_slots, alsub_server_t *out);

/*
 * Make a resident topology: build it (synchronously, on a stream of the server's own) and choose
 * how its frames are served:
 *   ALSUB_FRAMES_EVAL      the eval kernels on the cached topology (no operator is built);
 *   ALSUB_FRAMES_OPERATOR  one SpMV with the cached composite operator R (Sec. 3.6 "Single SpMV
 *                          evaluation"); falls back to EVAL when R does not fit the budget;
 *   ALSUB_FRAMES_FASTEST   build R, time one frame by each path and keep the faster;
 *   ALSUB_FRAMES_OPERATOR_MATRIX_FREE  alsub_apply_operator on a matrix-free operator
 *                          (ALSUB_OP_MATRIX_FREE): R's rows are the stencils the eval kernels
 *                          evaluate, so a frame costs what an EVAL frame costs and nothing but the
 *                          operator's scratch is stored.
 * Every resident also holds its frames' device input and output (12 V_0 + 12 V_L bytes, counted in
 * the budget): a frame copies its positions into them, runs there (a repeated frame replays the
 * topology's captured graph: one launch) and is copied out, so the frames of one resident run one
 * after another on the device while those of different residents overlap; a FRAME request itself
 * takes no device memory at admission.
 * Mesh arguments as alsub_mesh_create. *resident receives the id FRAME requests name.
 * Errors: those of the mesh, topology and operator calls, INVALID_ARG for an unknown mode, OOM when
 * the topology does not fit the budget.
 */
typedef enum {
    ALSUB_FRAMES_EVAL = 0,
    ALSUB_FRAMES_OPERATOR = 1,
    ALSUB_FRAMES_FASTEST = 2,
    ALSUB_FRAMES_OPERATOR_MATRIX_FREE = 3
} alsub_frame_path;

alsub_status alsub_serve_register(alsub_server_t server, alsub_scheme scheme, int32_t num_verts,
                                  int32_t num_faces, const int32_t *face_offsets_host,
                                  const int32_t *face_verts_host, int32_t num_creases,
                                  const int32_t *crease_verts_host, const float *crease_sharpness_host,
                                  int32_t levels, int32_t frame_path, int32_t *resident);

/* Queue a request; *ticket identifies it. The host arrays of the request are copied before
 * return. Errors: INVALID_ARG (bad request, unknown resident), UNSUPPORTED (counts), OOM (larger
 * than the budget left by the residents). Mesh validity is checked when the request runs and
 * reported in its result status. */
alsub_status alsub_serve_submit(alsub_server_t server, const alsub_request *request, uint64_t *ticket);

/* Wait up to timeout_us microseconds (0 = do not wait; at most 2^31 - 1) for a request. OK: done,
 * *result filled (result->status is the request's outcome). NOT_READY (timeout 0) or TIMEOUT:
 * still queued or in flight. INVALID_ARG: unknown ticket. */
alsub_status alsub_serve_poll(alsub_server_t server, uint64_t ticket, int32_t timeout_us,
                              alsub_result *result);

/* Forget a finished request and free the result the server kept for it. */
alsub_status alsub_serve_release(alsub_server_t server, uint64_t ticket);

/* paused != 0: admit nothing new (requests in flight finish, submitted ones wait); 0: resume. */
alsub_status alsub_serve_pause(alsub_server_t server, int32_t paused);

alsub_status alsub_serve_stats_get(alsub_server_t server, alsub_serve_stats *stats);

/* Stop the worker after the requests in flight finish (queued ones are dropped), free everything
 * the server holds, residents included. */
alsub_status alsub_serve_destroy(alsub_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* ALSUB_H */
