/*
 * AlSub oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial, FP64 half-edge subdivider that the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg use to check and time the CUDA path. Nothing in the product
 * library links, loads or calls it, and it shares no code, header or table with the CUDA path.
 *
 * It applies one level at a time with the CLASSICAL local rules (not the sparse-matrix form the
 * GPU uses), so that agreement between the two checks the paper's equivalence of both forms:
 *   Catmull-Clark  Sec. 3.1: face point (Eq. 1), edge point (Eq. 2), vertex update
 *                  (Eq. pos_update), topology refinement (step 4; the refined matrix layout of
 *                  Sec. 3.2 "Topology refinement": old vertices, then face point |v|+r, then edge
 *                  point |v|+|f|+e).
 *   Loop           Appendix B: edge point, smoothing Eq. loop_smooth with beta_n, 1-to-4 split.
 *   sqrt(3)        Appendix A: face point, smoothing Eq. sqrt2 with alpha_n (Eq. alpha),
 *                  one child triangle per corner (p_k, f_{F(l,k)}, f_i).
 *   Creases        Sec. 3.3: crease valency k (Eq. CC_crease_valency), vertex sharpness s
 *                  (Eq. CC_crease_vsharpness), Chaikin-style inheritance (Eqs. after Sec. 3.3's
 *                  two-step description). The vertex/edge crease rules themselves are delegated
 *                  by the paper to DeRose et al. 1998; the reading used here is:
 *                    edge point: sigma >= 1 -> midpoint; 0 < sigma < 1 -> (1-sigma) smooth +
 *                    sigma midpoint; vertex: k < 2 smooth; k == 2 sharp = (p_a + 6 p + p_b)/8;
 *                    k >= 3 sharp = p; result w sharp + (1-w) smooth, w = min(s, 1).
 *                  Chaikin neighbour of a crease end v: the other crease's sharpness when k(v)
 *                  == 2 and it is finite, else the crease's own sharpness. The inherited value
 *                  is evaluated in FP32, in the fixed order t = 3*s; u = s_o + t; w = u * 0.25;
 *                  y = w - 1; max(y, 0) (compile with -ffp-contract=off).
 *                  sqrt(3) (no crease treatment in the paper) keeps the infinitely sharp creases
 *                  as feature edges, handled as its boundaries are (below); finite sharpness is
 *                  ignored.
 *   Boundaries     Catmull-Clark (Sec. 3.1 "Boundaries", Eq. CC_boundary): an edge with one
 *                  face is a boundary edge; its edge point is its midpoint, and a boundary vertex
 *                  becomes 3/4 p + 1/8 (p_prev + p_next) with its two boundary neighbours. Every
 *                  other point follows the closed-mesh rules. A vertex on more than two boundary
 *                  edges (several fans) is non-manifold; a crease that touches a boundary vertex
 *                  is refused (the paper defines no combination). Loop (Appendix B gives no
 *                  boundary rule) takes the same two rules on its boundary, so that the boundary
 *                  is again the cubic B-spline curve of its control polygon. sqrt(3) (Appendix A
 *                  omits boundaries) follows Kobbelt 2000: feature edges (boundary edges and
 *                  infinitely sharp creases) are not flipped on the first step of each pair of
 *                  steps and are split into three on the second, their curves refined by the
 *                  ternary cubic B-spline masks (see sqrt3_level).
 * Edge numbering follows Sec. 3.2: edges are numbered in the order of the non-zeros of the upper
 * triangle of E, i.e. lexicographically by (min vertex, max vertex).
 * Child faces: face r with corners j = 0..c-1 is replaced by its children in corner order; the
 * child of corner j starts at the parent vertex v_j.
 *
 * Parity of the crease rule reading has no printed example in the paper: it is pinned only by its
 * limit cases (sigma = 0 smooth, sigma = inf cubic B-spline curve, sigma = 1 one sharp step).
 *
 * Patch mode (patch != 0, one level): the input is a patch cut out of a larger closed mesh, so
 * every scheme accepts its open edges and every point whose rule would need what lies beyond the
 * cut is NaN (an edge point of an open edge, a vertex point of a vertex on one, a sqrt(3) child
 * vertex across one is -1); a crease touching the cut is dropped and the vertex points of its ends
 * are NaN (their crease valency is unknown). All other points are exactly what the closed mesh
 * gives, which lets a test check sampled outputs of a mesh too large for the oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NONMANIFOLD = 2, OR_ERR_BOUNDARY = 3, OR_ERR_OOM = 4,
       OR_ERR_CREASE = 5 };
enum { OR_CC = 0, OR_LOOP = 1, OR_SQRT3 = 2 };

typedef struct {
    int V, F, nnz, E, K;
    int *off;          /* F+1 */
    int *fv;           /* nnz */
    double *P;         /* 3V */
    int *cv;           /* 2K crease endpoints */
    float *cs;         /* K crease sharpness */
    /* operator R_l mapping this level to the next (COO), if requested */
    long long rnnz;
    int *rr, *rc;
    double *rw;
} olevel;

typedef struct {
    int levels;
    olevel *L;         /* levels + 1 entries; entries not kept are left empty */
} oresult;

/* ---------------------------------------------------------------- half-edge view of a level */

typedef struct {
    int V, F, nnz;
    const int *off, *fv;
    int *cf;           /* corner -> face */
    int *nx, *pv;      /* next / previous corner in the face */
    int *tw;           /* twin corner (the corner running the other way along the edge) */
    int *vo, *vb;      /* outgoing corners bucketed by start vertex: vb[vo[v] .. vo[v+1]) */
    int *eid;          /* edge id per corner (lexicographic numbering) */
    int E;
    int *ea, *eb;      /* edge endpoints, ea < eb */
    int *eo;           /* a corner of each edge (the boundary corner of a boundary edge) */
    int B;             /* boundary corners (corners without a twin) */
    int patch;         /* patch mode: NaN instead of boundary rules */
    int *bo;           /* per vertex: its outgoing boundary corner, or -1 for an interior vertex */
} hedge;

static void hedge_free(hedge *h) {
    free(h->cf); free(h->nx); free(h->pv); free(h->tw); free(h->vo); free(h->vb);
    free(h->eid); free(h->ea); free(h->eb); free(h->eo); free(h->bo);
    memset(h, 0, sizeof(*h));
}

typedef struct { int a, b, c; } ekey;

static int ekey_cmp(const void *x, const void *y) {
    const ekey *p = (const ekey *)x, *q = (const ekey *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

/* Build corners, twins and the lexicographic edge numbering. 2-manifolds, closed unless
 * open != 0 (then a corner whose edge has no second face gets twin -1); open == 2 (a patch) also
 * accepts a vertex with several open fans (a pinch where the patch was cut). */
static int hedge_build(hedge *h, int V, int F, const int *off, const int *fv, int open) {
    memset(h, 0, sizeof(*h));
    h->V = V; h->F = F; h->nnz = off[F]; h->off = off; h->fv = fv;
    int n = h->nnz;
    h->cf = malloc(sizeof(int) * (size_t)n); h->nx = malloc(sizeof(int) * (size_t)n);
    h->pv = malloc(sizeof(int) * (size_t)n); h->tw = malloc(sizeof(int) * (size_t)n);
    h->vo = calloc((size_t)V + 1, sizeof(int)); h->vb = malloc(sizeof(int) * (size_t)n);
    h->eid = malloc(sizeof(int) * (size_t)n);
    h->bo = malloc(sizeof(int) * (size_t)V);
    if (!h->cf || !h->nx || !h->pv || !h->tw || !h->vo || !h->vb || !h->eid || !h->bo) return OR_ERR_OOM;
    for (int r = 0; r < F; r++) {
        int s = off[r], c = off[r + 1] - off[r];
        if (c < 3) return OR_ERR_ARG;
        for (int j = 0; j < c; j++) {
            h->cf[s + j] = r;
            h->nx[s + j] = s + (j + 1) % c;
            h->pv[s + j] = s + (j + c - 1) % c;
        }
    }
    for (int i = 0; i < n; i++) {
        if (fv[i] < 0 || fv[i] >= V) return OR_ERR_ARG;
        h->vo[fv[i] + 1]++;
    }
    for (int v = 0; v < V; v++) {
        if (h->vo[v + 1] == 0) return OR_ERR_ARG;    /* isolated vertex */
        h->vo[v + 1] += h->vo[v];
    }
    int *fill = calloc((size_t)V, sizeof(int));
    if (!fill) return OR_ERR_OOM;
    for (int i = 0; i < n; i++) h->vb[h->vo[fv[i]] + fill[fv[i]]++] = i;  /* ascending corners */
    free(fill);
    /* twin of a->b: the unique corner b->a */
    for (int i = 0; i < n; i++) {
        int a = fv[i], b = fv[h->nx[i]];
        if (a == b) return OR_ERR_ARG;
        int found = -1, cnt = 0;
        for (int q = h->vo[b]; q < h->vo[b + 1]; q++) {
            int d = h->vb[q];
            if (fv[h->nx[d]] == a) { found = d; cnt++; }
        }
        if (cnt == 0 && !open) return OR_ERR_BOUNDARY;
        if (cnt > 1) return OR_ERR_NONMANIFOLD;
        h->tw[i] = cnt ? found : -1;
        for (int q = h->vo[a]; q < h->vo[a + 1]; q++) {   /* duplicate directed edge */
            int d = h->vb[q];
            if (d != i && fv[h->nx[d]] == b) return OR_ERR_NONMANIFOLD;
        }
    }
    /* every vertex: its outgoing corners form a single fan. Interior vertex: one cycle under
     * x -> tw(pv(x)). Boundary vertex: exactly one outgoing boundary corner, where the chain under
     * the same step starts (no corner steps onto it) and which reaches every corner before it
     * ends at the incoming boundary edge. */
    h->B = 0;
    for (int v = 0; v < V; v++) {
        int deg = h->vo[v + 1] - h->vo[v], nb = 0, start = h->vb[h->vo[v]];
        for (int q = h->vo[v]; q < h->vo[v + 1]; q++)
            if (h->tw[h->vb[q]] < 0) { nb++; start = h->vb[q]; }
        h->bo[v] = nb ? start : -1;
        h->B += nb;
        if (nb > 1 && open == 2) continue;
        if (nb > 1) return OR_ERR_NONMANIFOLD;
        int x = start, steps = 0;
        if (nb == 0) {
            do { x = h->tw[h->pv[x]]; steps++; } while (x != start && steps <= deg);
        } else {
            steps = 1;
            while (h->tw[h->pv[x]] >= 0 && steps <= deg) { x = h->tw[h->pv[x]]; steps++; }
        }
        if (steps != deg) return OR_ERR_NONMANIFOLD;
    }
    /* edges: one per corner pair (or boundary corner); number them lexicographically by
     * (min, max) */
    if ((n + h->B) % 2) return OR_ERR_NONMANIFOLD;
    int E = (n + h->B) / 2;
    ekey *keys = malloc(sizeof(ekey) * (size_t)E);
    if (!keys) return OR_ERR_OOM;
    int k = 0;
    for (int i = 0; i < n; i++) {
        int a = fv[i], b = fv[h->nx[i]];
        if (h->tw[i] < 0 || a < b) {
            if (k == E) { free(keys); return OR_ERR_NONMANIFOLD; }
            keys[k].a = a < b ? a : b; keys[k].b = a < b ? b : a; keys[k].c = i; k++;
        }
    }
    if (k != E) { free(keys); return OR_ERR_NONMANIFOLD; }
    qsort(keys, (size_t)E, sizeof(ekey), ekey_cmp);
    h->E = E;
    h->ea = malloc(sizeof(int) * (size_t)E); h->eb = malloc(sizeof(int) * (size_t)E);
    h->eo = malloc(sizeof(int) * (size_t)E);
    if (!h->ea || !h->eb || !h->eo) { free(keys); return OR_ERR_OOM; }
    for (int e = 0; e < E; e++) {
        h->ea[e] = keys[e].a; h->eb[e] = keys[e].b; h->eo[e] = keys[e].c;
        h->eid[keys[e].c] = e;
        if (h->tw[keys[e].c] >= 0) h->eid[h->tw[keys[e].c]] = e;
    }
    free(keys);
    return OR_OK;
}

/* edge id of the undirected edge {a, b} or -1 (a boundary edge holds only one direction) */
static int hedge_find_edge(const hedge *h, int a, int b) {
    if (a < 0 || b < 0 || a >= h->V || b >= h->V) return -1;
    for (int t = 0; t < 2; t++) {
        int u = t ? b : a, w = t ? a : b;
        for (int q = h->vo[u]; q < h->vo[u + 1]; q++) {
            int d = h->vb[q];
            if (h->fv[h->nx[d]] == w) return h->eid[d];
        }
    }
    return -1;
}

/* ---------------------------------------------------------------- crease bookkeeping */

typedef struct {
    float *es;         /* sharpness per edge (0 = smooth) */
    int *k;            /* crease valency per vertex: incident edges with sigma > 0 */
    double *S;         /* sum of incident crease sharpness */
    int *n1, *n2;      /* the first two crease neighbours (for k == 2) */
    float *s1, *s2;    /* their crease sharpness */
    int *taint;        /* patch mode: the vertex lost a crease at the cut (its point is NaN) */
} creases;

static void creases_free(creases *c) {
    free(c->es); free(c->k); free(c->S); free(c->n1); free(c->n2); free(c->s1); free(c->s2); free(c->taint);
    memset(c, 0, sizeof(*c));
}

static int creases_build(creases *c, const hedge *h, int K, const int *cv, const float *cs) {
    memset(c, 0, sizeof(*c));
    c->es = calloc((size_t)h->E, sizeof(float));
    c->k = calloc((size_t)h->V, sizeof(int));
    c->S = calloc((size_t)h->V, sizeof(double));
    c->n1 = malloc(sizeof(int) * (size_t)h->V); c->n2 = malloc(sizeof(int) * (size_t)h->V);
    c->s1 = calloc((size_t)h->V, sizeof(float)); c->s2 = calloc((size_t)h->V, sizeof(float));
    c->taint = calloc((size_t)h->V, sizeof(int));
    if (!c->es || !c->k || !c->S || !c->n1 || !c->n2 || !c->s1 || !c->s2 || !c->taint) return OR_ERR_OOM;
    for (int i = 0; i < K; i++) {
        float s = cs[i];
        if (!(s >= 0.0f)) return OR_ERR_CREASE;        /* negative or NaN */
        int e = hedge_find_edge(h, cv[2 * i], cv[2 * i + 1]);
        if (e < 0 && h->patch && cv[2 * i] >= 0 && cv[2 * i] < h->V && cv[2 * i + 1] >= 0 && cv[2 * i + 1] < h->V) {
            c->taint[cv[2 * i]] = c->taint[cv[2 * i + 1]] = 1;   /* its faces lie beyond the cut */
            continue;
        }
        if (e < 0) return OR_ERR_CREASE;
        if (h->bo[cv[2 * i]] >= 0 || h->bo[cv[2 * i + 1]] >= 0) {
            if (!h->patch) return OR_ERR_BOUNDARY;
            c->taint[cv[2 * i]] = c->taint[cv[2 * i + 1]] = 1;
            continue;
        }
        if (c->es[e] != 0.0f) return OR_ERR_CREASE;    /* tagged twice */
        c->es[e] = s;
    }
    for (int v = 0; v < h->V; v++) { c->n1[v] = -1; c->n2[v] = -1; }
    for (int e = 0; e < h->E; e++) {
        float s = c->es[e];
        if (s > 0.0f) {
            int ends[2] = {h->ea[e], h->eb[e]};
            for (int t = 0; t < 2; t++) {
                int v = ends[t], o = ends[1 - t];
                if (c->k[v] == 0) { c->n1[v] = o; c->s1[v] = s; }
                else if (c->k[v] == 1) { c->n2[v] = o; c->s2[v] = s; }
                c->k[v]++;
                c->S[v] += (double)s;
            }
        }
    }
    return OR_OK;
}

/* Chaikin-style sharpness of the child half of crease (v, o) at end v, FP32 in a fixed order. */
static float chaikin_child(const creases *c, int v, int o, float s) {
    float so = s;
    if (c->k[v] == 2) {
        float other = (c->n1[v] == o) ? c->s2[v] : c->s1[v];
        if (isfinite(other)) so = other;
    }
    volatile float t = 3.0f * s;
    volatile float u = so + t;
    volatile float w = u * 0.25f;
    volatile float y = w - 1.0f;
    return y > 0.0f ? y : 0.0f;
}

/* crease-rule vertex: w sharp + (1-w) smooth for k >= 2 */
static void crease_vertex(const creases *c, const double *P, int v, double *out /* smooth in */) {
    int k = c->k[v];
    if (k < 2) return;
    double s = c->S[v] / (double)k;
    double w = s < 1.0 ? s : 1.0;
    double sharp[3];
    for (int d = 0; d < 3; d++) {
        if (k == 2) sharp[d] = (P[3 * c->n1[v] + d] + 6.0 * P[3 * v + d] + P[3 * c->n2[v] + d]) / 8.0;
        else sharp[d] = P[3 * v + d];
        out[d] = w * sharp[d] + (1.0 - w) * out[d];
    }
}

static void crease_edge(double sigma, const double *pa, const double *pb, double *out) {
    if (!(sigma > 0.0)) return;
    for (int d = 0; d < 3; d++) {
        double mid = 0.5 * (pa[d] + pb[d]);
        out[d] = sigma >= 1.0 ? mid : (1.0 - sigma) * out[d] + sigma * mid;
    }
}

/* ---------------------------------------------------------------- sparse row accumulator */

typedef struct { int n, cap; int *c; double *w; } row;

static int row_add(row *r, int col, double w) {
    for (int i = 0; i < r->n; i++) if (r->c[i] == col) { r->w[i] += w; return OR_OK; }
    if (r->n == r->cap) {
        int cap = r->cap ? 2 * r->cap : 64;
        int *c = realloc(r->c, sizeof(int) * (size_t)cap);
        if (!c) return OR_ERR_OOM;
        r->c = c;
        double *w2 = realloc(r->w, sizeof(double) * (size_t)cap);
        if (!w2) return OR_ERR_OOM;
        r->w = w2;
        r->cap = cap;
    }
    r->c[r->n] = col; r->w[r->n] = w; r->n++;
    return OR_OK;
}

typedef struct { long long n, cap; int *r, *c; double *w; } coo;

static int coo_push_row(coo *m, int rowi, row *r) {
    /* rows are emitted with columns ascending; exact zeros are dropped */
    for (int i = 1; i < r->n; i++) {
        int c = r->c[i]; double w = r->w[i]; int j = i - 1;
        while (j >= 0 && r->c[j] > c) { r->c[j + 1] = r->c[j]; r->w[j + 1] = r->w[j]; j--; }
        r->c[j + 1] = c; r->w[j + 1] = w;
    }
    for (int i = 0; i < r->n; i++) {
        if (r->w[i] == 0.0) continue;
        if (m->n == m->cap) {
            long long cap = m->cap ? 2 * m->cap : 1024;
            int *a = realloc(m->r, sizeof(int) * (size_t)cap); if (!a) return OR_ERR_OOM; m->r = a;
            int *b = realloc(m->c, sizeof(int) * (size_t)cap); if (!b) return OR_ERR_OOM; m->c = b;
            double *w = realloc(m->w, sizeof(double) * (size_t)cap); if (!w) return OR_ERR_OOM; m->w = w;
            m->cap = cap;
        }
        m->r[m->n] = rowi; m->c[m->n] = r->c[i]; m->w[m->n] = r->w[i]; m->n++;
    }
    r->n = 0;
    return OR_OK;
}

/* row += w * (crease-rule vertex row of v), applied as w_s * sharp + (1 - w_s) * smooth */
static int crease_vertex_row(const creases *c, int v, row *smooth) {
    int k = c->k[v];
    if (k < 2) return OR_OK;
    double s = c->S[v] / (double)k;
    double w = s < 1.0 ? s : 1.0;
    for (int i = 0; i < smooth->n; i++) smooth->w[i] *= (1.0 - w);
    int st;
    if (k == 2) {
        if ((st = row_add(smooth, c->n1[v], w / 8.0))) return st;
        if ((st = row_add(smooth, v, w * 6.0 / 8.0))) return st;
        if ((st = row_add(smooth, c->n2[v], w / 8.0))) return st;
    } else if ((st = row_add(smooth, v, w))) return st;
    return OR_OK;
}

static int crease_edge_row(double sigma, int a, int b, row *smooth) {
    if (!(sigma > 0.0)) return OR_OK;
    double w = sigma >= 1.0 ? 1.0 : sigma;
    for (int i = 0; i < smooth->n; i++) smooth->w[i] *= (1.0 - w);
    int st;
    if ((st = row_add(smooth, a, 0.5 * w))) return st;
    return row_add(smooth, b, 0.5 * w);
}

/* ---------------------------------------------------------------- one level of each scheme */

typedef struct {
    int V, F, nnz, K;
    int *off, *fv, *cv;
    float *cs;
    double *P;
} onext;

static int alloc_next(onext *o, int V, int F, int nnz, int Kmax) {
    o->V = V; o->F = F; o->nnz = nnz; o->K = 0;
    o->off = malloc(sizeof(int) * ((size_t)F + 1));
    o->fv = malloc(sizeof(int) * (size_t)nnz);
    o->P = malloc(sizeof(double) * 3 * (size_t)V);
    o->cv = malloc(sizeof(int) * 2 * ((size_t)Kmax + 1));
    o->cs = malloc(sizeof(float) * ((size_t)Kmax + 1));
    return (o->off && o->fv && o->P && o->cv && o->cs) ? OR_OK : OR_ERR_OOM;
}

static void push_crease(onext *o, int a, int b, float s) {
    if (s > 0.0f) { o->cv[2 * o->K] = a; o->cv[2 * o->K + 1] = b; o->cs[o->K] = s; o->K++; }
}

/* The two boundary neighbours of v: the end of its outgoing boundary edge (nb) and the start of
 * its incoming one (pb), found by walking the fan from the outgoing boundary corner to the corner
 * after which it ends. Returns 0 for an interior vertex. */
static int boundary_neighbours(const hedge *h, int v, int *nb, int *pb) {
    int x = h->bo[v];
    if (x < 0) return 0;
    *nb = h->fv[h->nx[x]];
    while (h->tw[h->pv[x]] >= 0) x = h->tw[h->pv[x]];
    *pb = h->fv[h->pv[x]];
    return 1;
}

/* Catmull-Clark, Sec. 3.1 classical rules. */
static int cc_level(const hedge *h, const creases *cr, const double *P, onext *o, coo *R) {
    int V = h->V, F = h->F, E = h->E, n = h->nnz;
    int st = alloc_next(o, V + F + E, n, 4 * n, 2 * E);
    if (st) return st;
    double *Pn = o->P;
    double *fp = Pn + 3 * (size_t)V;           /* face points: |v| + r */
    double *ep = Pn + 3 * ((size_t)V + F);     /* edge points: |v| + |f| + e */
    /* 1. face point: barycenter of the polygon (Eq. 1) */
    for (int r = 0; r < F; r++) {
        int s = h->off[r], c = h->off[r + 1] - s;
        for (int d = 0; d < 3; d++) {
            double acc = 0.0;
            for (int j = 0; j < c; j++) acc += P[3 * h->fv[s + j] + d];
            fp[3 * r + d] = acc / c;
        }
    }
    /* 2. edge point: (p_k + p_l + f_r + f_s) / 4 (Eq. 2), then the crease rule */
    for (int e = 0; e < E; e++) {
        int c0 = h->eo[e], c1 = h->tw[c0];
        int a = h->ea[e], b = h->eb[e], r = h->cf[c0];
        if (c1 < 0) {                              /* boundary edge: its midpoint */
            for (int d = 0; d < 3; d++) ep[3 * e + d] = h->patch ? NAN : 0.5 * (P[3 * a + d] + P[3 * b + d]);
            continue;
        }
        int s = h->cf[c1];
        for (int d = 0; d < 3; d++)
            ep[3 * e + d] = 0.25 * (P[3 * a + d] + P[3 * b + d] + fp[3 * r + d] + fp[3 * s + d]);
        if (cr) crease_edge((double)cr->es[e], P + 3 * a, P + 3 * b, ep + 3 * e);
    }
    /* 3. vertex update (Eq. pos_update):
     *    S(p) = 1/n ((n-3) p + 1/n sum f_j + 2/n sum (p + p_j)/2), then the crease rule */
    for (int v = 0; v < V; v++) {
        int nb, pb;
        if (boundary_neighbours(h, v, &nb, &pb)) {  /* Eq. CC_boundary */
            for (int d = 0; d < 3; d++)
                Pn[3 * v + d] = h->patch ? NAN : 0.75 * P[3 * v + d] + 0.125 * (P[3 * pb + d] + P[3 * nb + d]);
            continue;
        }
        int nv = h->vo[v + 1] - h->vo[v];
        double sf[3] = {0, 0, 0}, sm[3] = {0, 0, 0};
        for (int q = h->vo[v]; q < h->vo[v + 1]; q++) {
            int x = h->vb[q];                           /* corner v -> p_j in face f_j */
            int pj = h->fv[h->nx[x]], fj = h->cf[x];
            for (int d = 0; d < 3; d++) {
                sf[d] += fp[3 * fj + d];
                sm[d] += 0.5 * (P[3 * v + d] + P[3 * pj + d]);
            }
        }
        for (int d = 0; d < 3; d++)
            Pn[3 * v + d] = ((nv - 3) * P[3 * v + d] + sf[d] / nv + 2.0 * sm[d] / nv) / nv;
        if (cr) crease_vertex(cr, P, v, Pn + 3 * v);
        if (cr && cr->taint[v]) for (int d = 0; d < 3; d++) Pn[3 * v + d] = NAN;
    }
    /* 4. topology: face r -> c_r quads [v_j, e(j), f_r, e(j-1)] */
    for (int r = 0; r <= n; r++) o->off[r] = 4 * r;
    for (int x = 0; x < n; x++) {
        int r = h->cf[x];
        o->fv[4 * x + 0] = h->fv[x];
        o->fv[4 * x + 1] = V + F + h->eid[x];
        o->fv[4 * x + 2] = V + r;
        o->fv[4 * x + 3] = V + F + h->eid[h->pv[x]];
    }
    /* creases: both halves inherit a Chaikin-style sharpness */
    if (cr) {
        for (int e = 0; e < E; e++) {
            float s = cr->es[e];
            if (!(s > 0.0f)) continue;
            int a = h->ea[e], b = h->eb[e];
            push_crease(o, a, V + F + e, chaikin_child(cr, a, b, s));
            push_crease(o, V + F + e, b, chaikin_child(cr, b, a, s));
        }
    }
    /* operator rows, same rules as weights */
    if (R) {
        row rw = {0, 0, NULL, NULL};
        for (int v = 0; v < V && !st; v++) {
            int nb, pb;
            if (boundary_neighbours(h, v, &nb, &pb)) {
                st = row_add(&rw, v, 0.75);
                if (!st) st = row_add(&rw, pb, 0.125);
                if (!st) st = row_add(&rw, nb, 0.125);
                if (!st) st = coo_push_row(R, v, &rw);
                continue;
            }
            int nv = h->vo[v + 1] - h->vo[v];
            double inv2 = 1.0 / ((double)nv * nv);
            st = row_add(&rw, v, (nv - 3.0) / nv + 1.0 / nv);        /* (n-3)/n p + (n/n^2) p */
            for (int q = h->vo[v]; q < h->vo[v + 1] && !st; q++) {
                int x = h->vb[q], pj = h->fv[h->nx[x]], fj = h->cf[x];
                int s0 = h->off[fj], c = h->off[fj + 1] - s0;
                st = row_add(&rw, pj, inv2);
                for (int j = 0; j < c && !st; j++) st = row_add(&rw, h->fv[s0 + j], inv2 / c);
            }
            if (!st && cr) st = crease_vertex_row(cr, v, &rw);
            if (!st) st = coo_push_row(R, v, &rw);
        }
        for (int r = 0; r < F && !st; r++) {
            int s0 = h->off[r], c = h->off[r + 1] - s0;
            for (int j = 0; j < c && !st; j++) st = row_add(&rw, h->fv[s0 + j], 1.0 / c);
            if (!st) st = coo_push_row(R, V + r, &rw);
        }
        for (int e = 0; e < E && !st; e++) {
            int c0 = h->eo[e], c1 = h->tw[c0];
            if (c1 < 0) {
                st = row_add(&rw, h->ea[e], 0.5);
                if (!st) st = row_add(&rw, h->eb[e], 0.5);
                if (!st) st = coo_push_row(R, V + F + e, &rw);
                continue;
            }
            int fs[2] = {h->cf[c0], h->cf[c1]};
            st = row_add(&rw, h->ea[e], 0.25);
            if (!st) st = row_add(&rw, h->eb[e], 0.25);
            for (int t = 0; t < 2 && !st; t++) {
                int s0 = h->off[fs[t]], c = h->off[fs[t] + 1] - s0;
                for (int j = 0; j < c && !st; j++) st = row_add(&rw, h->fv[s0 + j], 0.25 / c);
            }
            if (!st && cr) st = crease_edge_row((double)cr->es[e], h->ea[e], h->eb[e], &rw);
            if (!st) st = coo_push_row(R, V + F + e, &rw);
        }
        free(rw.c); free(rw.w);
    }
    return st;
}

static double loop_beta(int n) {
    double t = 0.375 + 0.25 * cos(2.0 * M_PI / n);
    return (0.625 - t * t) / n;
}

/* Loop, Appendix B. */
static int loop_level(const hedge *h, const creases *cr, const double *P, onext *o, coo *R) {
    int V = h->V, F = h->F, E = h->E;
    int st = alloc_next(o, V + E, 4 * F, 12 * F, 2 * E);
    if (st) return st;
    double *Pn = o->P, *ep = Pn + 3 * (size_t)V;
    /* edge point: 3/8 (p_i + p_j) + 1/8 (p_k + p_l), k, l opposite (G(i,j), G(j,i)) */
    for (int e = 0; e < E; e++) {
        int c0 = h->eo[e], c1 = h->tw[c0];
        int a = h->ea[e], b = h->eb[e];
        if (c1 < 0) {                              /* boundary edge: its midpoint */
            for (int d = 0; d < 3; d++) ep[3 * e + d] = h->patch ? NAN : 0.5 * (P[3 * a + d] + P[3 * b + d]);
            continue;
        }
        int k = h->fv[h->pv[c0]], l = h->fv[h->pv[c1]];
        for (int d = 0; d < 3; d++)
            ep[3 * e + d] = 0.375 * (P[3 * a + d] + P[3 * b + d]) + 0.125 * (P[3 * k + d] + P[3 * l + d]);
        if (cr) crease_edge((double)cr->es[e], P + 3 * a, P + 3 * b, ep + 3 * e);
    }
    /* vertex: (1 - n beta) p + beta sum p_j (Eq. loop_smooth); a boundary vertex as in
     * Eq. CC_boundary */
    for (int v = 0; v < V; v++) {
        int nb, pb;
        if (boundary_neighbours(h, v, &nb, &pb)) {
            for (int d = 0; d < 3; d++)
                Pn[3 * v + d] = h->patch ? NAN : 0.75 * P[3 * v + d] + 0.125 * (P[3 * pb + d] + P[3 * nb + d]);
            continue;
        }
        int nv = h->vo[v + 1] - h->vo[v];
        double beta = loop_beta(nv), sm[3] = {0, 0, 0};
        for (int q = h->vo[v]; q < h->vo[v + 1]; q++) {
            int pj = h->fv[h->nx[h->vb[q]]];
            for (int d = 0; d < 3; d++) sm[d] += P[3 * pj + d];
        }
        for (int d = 0; d < 3; d++) Pn[3 * v + d] = (1.0 - nv * beta) * P[3 * v + d] + beta * sm[d];
        if (cr) crease_vertex(cr, P, v, Pn + 3 * v);
        if (cr && cr->taint[v]) for (int d = 0; d < 3; d++) Pn[3 * v + d] = NAN;
    }
    /* topology: triangle (p_k, p_l, p_m) -> three corner triangles and the centre one */
    for (int r = 0; r <= 4 * F; r++) o->off[r] = 3 * r;
    for (int r = 0; r < F; r++) {
        int s = h->off[r];
        int e0 = V + h->eid[s], e1 = V + h->eid[s + 1], e2 = V + h->eid[s + 2];
        int v0 = h->fv[s], v1 = h->fv[s + 1], v2 = h->fv[s + 2];
        int *t = o->fv + 12 * (size_t)r;
        t[0] = v0; t[1] = e0; t[2] = e2;
        t[3] = v1; t[4] = e1; t[5] = e0;
        t[6] = v2; t[7] = e2; t[8] = e1;
        t[9] = e0; t[10] = e1; t[11] = e2;
    }
    if (cr) {
        for (int e = 0; e < E; e++) {
            float s = cr->es[e];
            if (!(s > 0.0f)) continue;
            int a = h->ea[e], b = h->eb[e];
            push_crease(o, a, V + e, chaikin_child(cr, a, b, s));
            push_crease(o, V + e, b, chaikin_child(cr, b, a, s));
        }
    }
    if (R) {
        row rw = {0, 0, NULL, NULL};
        for (int v = 0; v < V && !st; v++) {
            int nb, pb;
            if (boundary_neighbours(h, v, &nb, &pb)) {
                st = row_add(&rw, v, 0.75);
                if (!st) st = row_add(&rw, pb, 0.125);
                if (!st) st = row_add(&rw, nb, 0.125);
                if (!st) st = coo_push_row(R, v, &rw);
                continue;
            }
            int nv = h->vo[v + 1] - h->vo[v];
            double beta = loop_beta(nv);
            st = row_add(&rw, v, 1.0 - nv * beta);
            for (int q = h->vo[v]; q < h->vo[v + 1] && !st; q++)
                st = row_add(&rw, h->fv[h->nx[h->vb[q]]], beta);
            if (!st && cr) st = crease_vertex_row(cr, v, &rw);
            if (!st) st = coo_push_row(R, v, &rw);
        }
        for (int e = 0; e < E && !st; e++) {
            int c0 = h->eo[e], c1 = h->tw[c0];
            if (c1 < 0) {
                st = row_add(&rw, h->ea[e], 0.5);
                if (!st) st = row_add(&rw, h->eb[e], 0.5);
                if (!st) st = coo_push_row(R, V + e, &rw);
                continue;
            }
            st = row_add(&rw, h->ea[e], 0.375);
            if (!st) st = row_add(&rw, h->eb[e], 0.375);
            if (!st) st = row_add(&rw, h->fv[h->pv[c0]], 0.125);
            if (!st) st = row_add(&rw, h->fv[h->pv[c1]], 0.125);
            if (!st && cr) st = crease_edge_row((double)cr->es[e], h->ea[e], h->eb[e], &rw);
            if (!st) st = coo_push_row(R, V + e, &rw);
        }
        free(rw.c); free(rw.w);
    }
    return st;
}

static double sqrt3_alpha(int n) { return (4.0 - 2.0 * cos(2.0 * M_PI / n)) / 9.0; }

/* sqrt(3), Appendix A, with feature edges: the boundary edges and the infinitely sharp creases
 * (the paper omits both; the treatment follows Kobbelt 2000, Sec. 4 "Boundaries"). Refinement
 * alternates between two kinds of step:
 *   first step of a pair (odd, from an even level): a face point f_i for every triangle; every
 *     edge but the feature edges is flipped, so corner k of triangle i = (k, l, m) gives
 *     (p_k, f_{F(l,k)}, f_i), or (p_k, p_l, f_i) when k -> l is a feature edge; vertices on
 *     feature curves (two feature edges) and corners (three or more) keep their positions;
 *   second step (even, from an odd level): every triangle with a feature edge a -> b (exactly one,
 *     by construction of the first step) gets no face point; the edge is split into three by two
 *     new points q1 (near a) and q2 (near b), and the triangle (a, b, c) into (a, q1, c),
 *     (q1, q2, c), (q2, b, c); an edge flips only between two triangles with face points; the
 *     feature curve is refined by the ternary cubic B-spline masks (1, 16, 10)/27, (10, 16, 1)/27
 *     for q1, q2 and (4, 19, 4)/27 for its vertices, a curve end (a corner or a dart) being
 *     mirrored (its neighbour beyond it read as 2 p - p_next, which makes the points next to it
 *     the linear thirds); corners stay fixed.
 * Every other vertex takes the smooth rule (Eq. sqrt2), darts (one feature edge) included.
 * Numbering: old vertices, then slot |v| + i of triangle i (its face point, or the point of its
 * feature edge nearer the edge's start), then |v| + |f| + b for the second point of the b-th
 * boundary edge (in edge order). feat: per edge, 1 for a feature edge; ff: per vertex, its feature
 * valency and its feature neighbours (the two first found). */
typedef struct { int k, n1, n2; } fvert;

static void fvert_add(fvert *fvx, int v, int o) {
    if (fvx[v].k == 0) fvx[v].n1 = o;
    else if (fvx[v].k == 1) fvx[v].n2 = o;
    fvx[v].k++;
}

static int sqrt3_level(const hedge *h, const creases *cr, const double *P, int odd, onext *o, coo *R) {
    int V = h->V, F = h->F, E = h->E;
    int *feat = calloc((size_t)E, sizeof(int)), *brank = malloc(sizeof(int) * (size_t)E);
    fvert *fx = calloc((size_t)V, sizeof(fvert));
    int *fcorner = malloc(sizeof(int) * (size_t)F);          /* the triangle's feature corner, or -1 */
    if (!feat || !brank || !fx || !fcorner) { free(feat); free(brank); free(fx); free(fcorner); return OR_ERR_OOM; }
    int nb = 0, nfeat = 0;
    /* boundary edges ranked in corner order (a boundary edge has one corner); in patch mode the cut
     * is no feature: what lies across it is unknown (-1, NaN) */
    for (int e = 0; e < E; e++) brank[e] = -1;
    for (int x = 0; x < h->nnz; x++)
        if (h->tw[x] < 0 && !h->patch) brank[h->eid[x]] = nb++;
    for (int e = 0; e < E; e++) {
        int boundary = h->tw[h->eo[e]] < 0 && !h->patch;
        int crease = cr && cr->es && isinf(cr->es[e]);
        if (boundary || crease) {
            feat[e] = 1;
            nfeat++;
            fvert_add(fx, h->ea[e], h->eb[e]);
            fvert_add(fx, h->eb[e], h->ea[e]);
        }
    }
    int st = OR_OK;
    for (int r = 0; r < F && !st; r++) {
        fcorner[r] = -1;
        for (int j = 0; j < 3; j++) {
            int x = h->off[r] + j;
            if (!feat[h->eid[x]]) continue;
            if (!odd && fcorner[r] >= 0) st = OR_ERR_ARG;      /* cannot follow a first step */
            fcorner[r] = x;
        }
    }
    if (!st) st = alloc_next(o, V + F + (odd ? 0 : nb), 3 * F, 9 * F, odd ? nfeat : 3 * nfeat);
    if (st) { free(feat); free(brank); free(fx); free(fcorner); return st; }
    double *Pn = o->P;
    /* the neighbour of feature vertex v beyond it, seen from its feature neighbour w */
    /* face points (every triangle on a first step, the triangles without a feature edge on a
     * second one) */
    for (int r = 0; r < F; r++) {
        if (!odd && fcorner[r] >= 0) continue;
        int s = h->off[r];
        for (int d = 0; d < 3; d++)
            Pn[3 * (V + r) + d] = (P[3 * h->fv[s] + d] + P[3 * h->fv[s + 1] + d] + P[3 * h->fv[s + 2] + d]) / 3.0;
    }
    /* vertex points */
    for (int v = 0; v < V; v++) {
        const double *p = P + 3 * v;
        double *q = Pn + 3 * v;
        int k = fx[v].k;
        if (k >= 3 || (odd && k == 2)) {                    /* corner, or a curve on a first step */
            for (int d = 0; d < 3; d++) q[d] = p[d];
        } else if (k == 2) {                                 /* curve vertex, second step */
            const double *a = P + 3 * fx[v].n1, *b = P + 3 * fx[v].n2;
            for (int d = 0; d < 3; d++) q[d] = (4.0 * a[d] + 19.0 * p[d] + 4.0 * b[d]) / 27.0;
        } else {                                             /* S(p) = (1 - alpha) p + alpha / n sum p_j */
            int nv = h->vo[v + 1] - h->vo[v];
            double al = sqrt3_alpha(nv), sm[3] = {0, 0, 0};
            for (int qq = h->vo[v]; qq < h->vo[v + 1]; qq++) {
                int pj = h->fv[h->nx[h->vb[qq]]];
                for (int d = 0; d < 3; d++) sm[d] += P[3 * pj + d];
            }
            for (int d = 0; d < 3; d++) q[d] = (1.0 - al) * p[d] + al / nv * sm[d];
        }
        if (h->patch && h->bo[v] >= 0) for (int d = 0; d < 3; d++) q[d] = NAN;
    }
    /* second step: the two points of every feature edge */
    if (!odd) {
        for (int e = 0; e < E; e++) {
            if (!feat[e]) continue;
            int x = h->eo[e], a = h->fv[x], b = h->fv[h->nx[x]];
            int sa = V + h->cf[x];                                          /* near a */
            int sb = h->tw[x] < 0 ? V + F + brank[e] : V + h->cf[h->tw[x]]; /* near b */
            double pa_beyond[3], pb_beyond[3];
            for (int d = 0; d < 3; d++) {
                int wa = fx[a].k == 2 ? (fx[a].n1 == b ? fx[a].n2 : fx[a].n1) : -1;
                int wb = fx[b].k == 2 ? (fx[b].n1 == a ? fx[b].n2 : fx[b].n1) : -1;
                pa_beyond[d] = wa >= 0 ? P[3 * wa + d] : 2.0 * P[3 * a + d] - P[3 * b + d];
                pb_beyond[d] = wb >= 0 ? P[3 * wb + d] : 2.0 * P[3 * b + d] - P[3 * a + d];
            }
            for (int d = 0; d < 3; d++) {
                Pn[3 * sa + d] = (pa_beyond[d] + 16.0 * P[3 * a + d] + 10.0 * P[3 * b + d]) / 27.0;
                Pn[3 * sb + d] = (10.0 * P[3 * a + d] + 16.0 * P[3 * b + d] + pb_beyond[d]) / 27.0;
            }
        }
    }
    /* children */
    for (int r = 0; r <= 3 * F; r++) o->off[r] = 3 * r;
    for (int r = 0; r < F; r++) {
        int s = h->off[r];
        if (!odd && fcorner[r] >= 0) {
            int x = fcorner[r], e = h->eid[x];
            int a = h->fv[x], b = h->fv[h->nx[x]], c = h->fv[h->pv[x]];
            int q1 = V + r, q2 = h->tw[x] < 0 ? V + F + brank[e] : V + h->cf[h->tw[x]];
            int ch[9] = {a, q1, c, q1, q2, c, q2, b, c};
            memcpy(o->fv + 9 * r, ch, sizeof(ch));
            continue;
        }
        for (int j = 0; j < 3; j++) {
            int x = s + j, t = h->tw[x];
            /* flipped when neither side is a feature: the edge is no feature and, on a second
             * step, the triangle across it has a face point */
            if (t < 0 && !feat[h->eid[x]]) {                 /* patch mode: across the cut */
                o->fv[3 * x + 0] = h->fv[x];
                o->fv[3 * x + 1] = -1;
                o->fv[3 * x + 2] = V + r;
                continue;
            }
            int flip = !feat[h->eid[x]] && (odd || fcorner[h->cf[t]] < 0);
            o->fv[3 * x + 0] = h->fv[x];
            o->fv[3 * x + 1] = flip ? V + h->cf[t] : h->fv[h->nx[x]];
            o->fv[3 * x + 2] = V + r;
        }
    }
    /* crease edges of the next level (boundaries need no list) */
    for (int e = 0; e < E; e++) {
        if (!feat[e] || h->tw[h->eo[e]] < 0) continue;
        int x = h->eo[e], a = h->fv[x], b = h->fv[h->nx[x]];
        if (odd) {
            push_crease(o, a, b, INFINITY);
        } else {
            int q1 = V + h->cf[x], q2 = V + h->cf[h->tw[x]];
            push_crease(o, a, q1, INFINITY);
            push_crease(o, q1, q2, INFINITY);
            push_crease(o, q2, b, INFINITY);
        }
    }
    if (R) {
        row rw = {0, 0, NULL, NULL};
        for (int v = 0; v < V && !st; v++) {
            int k = fx[v].k;
            if (k >= 3 || (odd && k == 2)) {
                st = row_add(&rw, v, 1.0);
            } else if (k == 2) {
                st = row_add(&rw, fx[v].n1, 4.0 / 27.0);
                if (!st) st = row_add(&rw, v, 19.0 / 27.0);
                if (!st) st = row_add(&rw, fx[v].n2, 4.0 / 27.0);
            } else {
                int nv = h->vo[v + 1] - h->vo[v];
                double al = sqrt3_alpha(nv);
                st = row_add(&rw, v, 1.0 - al);
                for (int qq = h->vo[v]; qq < h->vo[v + 1] && !st; qq++)
                    st = row_add(&rw, h->fv[h->nx[h->vb[qq]]], al / nv);
            }
            if (!st) st = coo_push_row(R, v, &rw);
        }
        for (int r = 0; r < F && !st; r++) {
            if (!odd && fcorner[r] >= 0) continue;
            int s = h->off[r];
            for (int j = 0; j < 3 && !st; j++) st = row_add(&rw, h->fv[s + j], 1.0 / 3.0);
            if (!st) st = coo_push_row(R, V + r, &rw);
        }
        for (int e = 0; e < E && !st && !odd; e++) {
            if (!feat[e]) continue;
            int x = h->eo[e], a = h->fv[x], b = h->fv[h->nx[x]];
            int sa = V + h->cf[x];
            int sb = h->tw[x] < 0 ? V + F + brank[e] : V + h->cf[h->tw[x]];
            int wa = fx[a].k == 2 ? (fx[a].n1 == b ? fx[a].n2 : fx[a].n1) : -1;
            int wb = fx[b].k == 2 ? (fx[b].n1 == a ? fx[b].n2 : fx[b].n1) : -1;
            /* q1 = (beyond_a + 16 a + 10 b) / 27 with beyond_a = 2 a - b at a curve end */
            if (wa >= 0) { st = row_add(&rw, wa, 1.0 / 27.0); if (!st) st = row_add(&rw, a, 16.0 / 27.0); if (!st) st = row_add(&rw, b, 10.0 / 27.0); }
            else { st = row_add(&rw, a, 18.0 / 27.0); if (!st) st = row_add(&rw, b, 9.0 / 27.0); }
            if (!st) st = coo_push_row(R, sa, &rw);
            if (st) break;
            if (wb >= 0) { st = row_add(&rw, a, 10.0 / 27.0); if (!st) st = row_add(&rw, b, 16.0 / 27.0); if (!st) st = row_add(&rw, wb, 1.0 / 27.0); }
            else { st = row_add(&rw, a, 9.0 / 27.0); if (!st) st = row_add(&rw, b, 18.0 / 27.0); }
            if (!st) st = coo_push_row(R, sb, &rw);
        }
        free(rw.c); free(rw.w);
    }
    free(feat); free(brank); free(fx); free(fcorner);
    return st;
}

/* ---------------------------------------------------------------- driver and accessors */

static void level_free(olevel *l) {
    free(l->off); free(l->fv); free(l->P); free(l->cv); free(l->cs);
    free(l->rr); free(l->rc); free(l->rw);
    memset(l, 0, sizeof(*l));
}

void or_free(oresult *r) {
    if (!r) return;
    for (int l = 0; l <= r->levels; l++) level_free(&r->L[l]);
    free(r->L);
    free(r);
}

/*
 * Refine `levels` times. keep_all = 0 keeps only the last level; want_operator = 1 stores the
 * operator R_l of every kept level l < levels (COO, FP64). start_level: the level the input is at
 * (it decides which kind of sqrt(3) step comes first).
 */
int or_run(int scheme, int levels, int keep_all, int want_operator, int patch, int start_level,
           int V, int F, const int *off, const int *fv, const double *P0,
           int K, const int *cv, const float *cs, oresult **out) {
    *out = NULL;
    if (scheme < 0 || scheme > 2 || levels < 0 || V <= 0 || F <= 0 || K < 0) return OR_ERR_ARG;
    if (patch && (levels != 1 || want_operator)) return OR_ERR_ARG;
    if (off[0] != 0) return OR_ERR_ARG;
    for (int r = 0; r < F; r++) {
        int c = off[r + 1] - off[r];
        if (c < 3 || (scheme != OR_CC && c != 3)) return OR_ERR_ARG;
    }
    oresult *res = calloc(1, sizeof(oresult));
    if (!res) return OR_ERR_OOM;
    res->levels = levels;
    res->L = calloc((size_t)levels + 1, sizeof(olevel));
    if (!res->L) { free(res); return OR_ERR_OOM; }
    /* level 0: copy the input; sigma = 0 creases carry nothing and are dropped */
    olevel *cur = &res->L[0];
    cur->V = V; cur->F = F; cur->nnz = off[F];
    cur->off = malloc(sizeof(int) * ((size_t)F + 1)); cur->fv = malloc(sizeof(int) * (size_t)off[F]);
    cur->P = malloc(sizeof(double) * 3 * (size_t)V);
    cur->cv = malloc(sizeof(int) * 2 * ((size_t)K + 1)); cur->cs = malloc(sizeof(float) * ((size_t)K + 1));
    if (!cur->off || !cur->fv || !cur->P || !cur->cv || !cur->cs) { or_free(res); return OR_ERR_OOM; }
    memcpy(cur->off, off, sizeof(int) * ((size_t)F + 1));
    memcpy(cur->fv, fv, sizeof(int) * (size_t)off[F]);
    memcpy(cur->P, P0, sizeof(double) * 3 * (size_t)V);
    cur->K = 0;
    {
        for (int i = 0; i < K; i++) {
            if (!(cs[i] >= 0.0f)) { or_free(res); return OR_ERR_CREASE; }
            /* sqrt(3) keeps the infinitely sharp creases only (feature edges) */
            if (cs[i] > 0.0f && (scheme != OR_SQRT3 || isinf(cs[i]))) {
                cur->cv[2 * cur->K] = cv[2 * i]; cur->cv[2 * cur->K + 1] = cv[2 * i + 1];
                cur->cs[cur->K] = cs[i]; cur->K++;
            }
        }
    }
    int st = OR_OK;
    int last = 0;
    for (int l = 0; l <= levels && !st; l++) {
        olevel *L = &res->L[last];
        if (patch && l == levels) break;          /* a patch's child may reference the cut (-1) */
        hedge h;
        st = hedge_build(&h, L->V, L->F, L->off, L->fv, patch ? 2 : 1);
        h.patch = patch;
        if (st) { hedge_free(&h); break; }
        L->E = h.E;
        creases cr;
        memset(&cr, 0, sizeof(cr));
        int use_cr = L->K > 0;
        if (use_cr) st = creases_build(&cr, &h, L->K, L->cv, L->cs);
        if (st || l == levels) { creases_free(&cr); hedge_free(&h); break; }
        onext o;
        memset(&o, 0, sizeof(o));
        coo R = {0, 0, NULL, NULL, NULL};
        coo *Rp = want_operator ? &R : NULL;
        if (scheme == OR_CC) st = cc_level(&h, use_cr ? &cr : NULL, L->P, &o, Rp);
        else if (scheme == OR_LOOP) st = loop_level(&h, use_cr ? &cr : NULL, L->P, &o, Rp);
        else st = sqrt3_level(&h, use_cr ? &cr : NULL, L->P, ((l + start_level) & 1) == 0, &o, Rp);
        creases_free(&cr);
        hedge_free(&h);
        if (Rp) { L->rnnz = R.n; L->rr = R.r; L->rc = R.c; L->rw = R.w; }
        olevel *N = &res->L[l + 1];
        N->V = o.V; N->F = o.F; N->nnz = o.nnz; N->K = o.K;
        N->off = o.off; N->fv = o.fv; N->P = o.P; N->cv = o.cv; N->cs = o.cs;
        if (st) break;
        if (!keep_all) level_free(L);
        last = l + 1;
    }
    if (st) { or_free(res); return st; }
    *out = res;
    return OR_OK;
}

static const olevel *lev(const oresult *r, int l) {
    if (!r || l < 0 || l > r->levels || !r->L[l].off) return NULL;
    return &r->L[l];
}

/* V, F, nnz, E, K, rnnz of a kept level */
int or_counts(const oresult *r, int l, long long *outv) {
    const olevel *L = lev(r, l);
    if (!L) return OR_ERR_ARG;
    outv[0] = L->V; outv[1] = L->F; outv[2] = L->nnz; outv[3] = L->E; outv[4] = L->K; outv[5] = L->rnnz;
    return OR_OK;
}

int or_faces(const oresult *r, int l, int *off, int *fv) {
    const olevel *L = lev(r, l);
    if (!L) return OR_ERR_ARG;
    memcpy(off, L->off, sizeof(int) * ((size_t)L->F + 1));
    memcpy(fv, L->fv, sizeof(int) * (size_t)L->nnz);
    return OR_OK;
}

int or_positions(const oresult *r, int l, double *P) {
    const olevel *L = lev(r, l);
    if (!L) return OR_ERR_ARG;
    memcpy(P, L->P, sizeof(double) * 3 * (size_t)L->V);
    return OR_OK;
}

int or_creases(const oresult *r, int l, int *cv, float *cs) {
    const olevel *L = lev(r, l);
    if (!L) return OR_ERR_ARG;
    memcpy(cv, L->cv, sizeof(int) * 2 * (size_t)L->K);
    memcpy(cs, L->cs, sizeof(float) * (size_t)L->K);
    return OR_OK;
}

int or_operator(const oresult *r, int l, int *rows, int *cols, double *w) {
    const olevel *L = lev(r, l);
    if (!L || !L->rr) return OR_ERR_ARG;
    memcpy(rows, L->rr, sizeof(int) * (size_t)L->rnnz);
    memcpy(cols, L->rc, sizeof(int) * (size_t)L->rnnz);
    memcpy(w, L->rw, sizeof(double) * (size_t)L->rnnz);
    return OR_OK;
}
