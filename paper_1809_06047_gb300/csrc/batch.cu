// Ragged batches: vertex refinement of many built topologies of uneven sizes (and any mix of
// schemes and level counts) with one launch per level per kernel class. Level l of every member
// that has it forms one flattened work list of face tiles (closed-form sizes, so the plan is
// fixed when the batch is made); the whole batched call is captured once into a CUDA graph and
// replayed. Block size and grid persistence are chosen by alsub_batch_tune, which times the
// candidates on the batch itself.
#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace alsub;

struct alsub_batch_s {
    std::vector<TopoImpl *> T;
    std::vector<const float *> P0;
    std::vector<float *> PL;
    int maxL = 0;
    int block = 256;
    int blocks_per_sm = 4;          // persistent grid = SMs x this; 0 = one CTA per tile
    int sms = 152;
    std::vector<std::vector<BatchClass>> cc, tri;   // per level
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    long long launches = 0;
    int per_call = 0;               // kernels one batched call launches
};

namespace {

void free_plans(alsub_batch_s &B) {
    for (auto *v : {&B.cc, &B.tri})
        for (auto &lv : *v)
            for (BatchClass &c : lv) {
                cudaFree(c.args);
                cudaFree(c.tile_begin);
            }
    B.cc.clear();
    B.tri.clear();
}

void drop_graph(alsub_batch_s &B) {
    if (B.exec) cudaGraphExecDestroy(B.exec);
    if (B.graph) cudaGraphDestroy(B.graph);
    B.exec = nullptr;
    B.graph = nullptr;
}

// positions of member i on the input / output side of level l
void member_buffers(const alsub_batch_s &B, int i, int l, const float **in, float **out) {
    const TopoImpl &T = *B.T[i];
    const size_t half = T.scratch_bytes / (2 * sizeof(float));
    *in = l == 0 ? B.P0[i] : T.scratch + half * ((l - 1) & 1);
    *out = l == T.levels - 1 ? B.PL[i] : T.scratch + half * (l & 1);
}

alsub_status replan(alsub_batch_s &B) {
    drop_graph(B);
    free_plans(B);
    B.cc.resize(B.maxL);
    B.tri.resize(B.maxL);
    for (int l = 0; l < B.maxL; l++) {
        std::vector<EvalItem> icc, itri;
        for (size_t i = 0; i < B.T.size(); i++) {
            if (l >= B.T[i]->levels) continue;
            EvalItem it{B.T[i], l, nullptr, nullptr};
            float *o;
            member_buffers(B, (int)i, l, &it.P, &o);
            it.Pn = o;
            (B.T[i]->scheme == ALSUB_CATMULL_CLARK ? icc : itri).push_back(it);
        }
        if (!icc.empty()) B.cc[l] = cc_batch_plan(icc, B.block);
        if (!itri.empty()) B.tri[l] = tri_batch_plan(itri, B.block);
        for (auto *v : {&B.cc[l], &B.tri[l]})
            for (const BatchClass &c : *v)
                if (c.tiles < 0) return report(ALSUB_ERR_OOM, "batch plan: device allocation failed");
    }
    return ALSUB_OK;
}

int enqueue(alsub_batch_s &B, cudaStream_t s) {
    int k = 0;
    const int grid = B.blocks_per_sm > 0 ? B.sms * B.blocks_per_sm : 0x7fffffff;
    for (size_t i = 0; i < B.T.size(); i++)
        if (B.T[i]->levels == 0)
            cudaMemcpyAsync(B.PL[i], B.P0[i], sizeof(float) * 3 * (size_t)B.T[i]->L[0].V,
                            cudaMemcpyDeviceToDevice, s);
    for (int l = 0; l < B.maxL; l++) {
        for (const BatchClass &c : B.cc[l]) { cc_batch_launch(c, B.block, grid, s); k++; }
        for (const BatchClass &c : B.tri[l]) { tri_batch_launch(c, B.block, grid, s); k++; }
        for (size_t i = 0; i < B.T.size(); i++) {
            TopoImpl &T = *B.T[i];
            if (l >= T.levels) continue;
            const bool fix = crease_alive(T, l);
            const bool ed = l + 1 < (int)T.edits.size() && T.edits[l + 1].n > 0;
            if (!fix && !ed) continue;
            const float *in;
            float *out;
            member_buffers(B, (int)i, l, &in, &out);
            if (fix) { crease_fix(T, l, in, out, s); k++; }
            if (ed) { apply_edits(T, l + 1, out, s); k++; }
        }
    }
    return k;
}

alsub_status run(alsub_batch_s &B, cudaStream_t s) {
    if (!s) {  // the legacy stream cannot be captured: plain launches
        B.per_call = enqueue(B, s);
    } else {
        if (B.exec && B.graph_stream != s) drop_graph(B);
        if (!B.exec) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return report(ALSUB_ERR_DEVICE, "batch: stream capture failed to start");
            B.per_call = enqueue(B, s);
            if (cudaStreamEndCapture(s, &g) != cudaSuccess || !g) {
                cudaGetLastError();
                return report(ALSUB_ERR_DEVICE, "batch: stream capture failed");
            }
            if (cudaGraphInstantiate(&B.exec, g, 0) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphDestroy(g);
                return report(ALSUB_ERR_DEVICE, "batch: graph instantiation failed");
            }
            B.graph = g;
            B.graph_stream = s;
        }
        if (cudaGraphLaunch(B.exec, s) != cudaSuccess) {
            cudaGetLastError();
            return report(ALSUB_ERR_DEVICE, "batch: graph launch failed");
        }
    }
    B.launches += B.per_call;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ALSUB_OK : report(ALSUB_ERR_DEVICE, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

alsub_status alsub_batch_create(int32_t n, const alsub_topology_t *topos, const float *const *P0_dev,
                                float *const *PL_dev, alsub_batch_t *out) {
    if (!out || n <= 0 || !topos || !P0_dev || !PL_dev) return report(ALSUB_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    alsub_batch_s *B = new (std::nothrow) alsub_batch_s();
    if (!B) return report(ALSUB_ERR_OOM, "host allocation failed");
    for (int i = 0; i < n; i++) {
        if (!topos[i] || !P0_dev[i] || !PL_dev[i]) { delete B; return report(ALSUB_ERR_INVALID_ARG, "NULL member"); }
        TopoImpl *T = topology_impl(topos[i]);
        if (!T->built) { delete B; return report(ALSUB_ERR_INVALID_ARG, "batch member topology not built"); }
        if (T->mesh->B > 0) {
            delete B;
            return report(ALSUB_ERR_UNSUPPORTED, "batch members must be closed meshes (no boundary repair)");
        }
        if (T->s3f) {
            delete B;
            return report(ALSUB_ERR_UNSUPPORTED, "batch members: a sqrt(3) mesh with infinitely sharp creases takes "
                                                 "the general feature path, which is not batched");
        }
        for (TopoImpl *U : B->T)
            if (U == T) { delete B; return report(ALSUB_ERR_INVALID_ARG, "a topology appears twice in the batch"); }
        B->T.push_back(T);
        B->P0.push_back(P0_dev[i]);
        B->PL.push_back(PL_dev[i]);
        B->maxL = std::max(B->maxL, T->levels);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev);
    alsub_status st = replan(*B);
    if (st) { free_plans(*B); delete B; return st; }
    *out = B;
    return ALSUB_OK;
}

alsub_status alsub_batch_configure(alsub_batch_t b, int32_t block, int32_t blocks_per_sm) {
    if (!b || (block != 128 && block != 256 && block != 512) || blocks_per_sm < 0 || blocks_per_sm > 16)
        return report(ALSUB_ERR_INVALID_ARG, "block must be 128, 256 or 512; blocks_per_sm 0..16");
    cudaDeviceSynchronize();
    b->block = block;
    b->blocks_per_sm = blocks_per_sm;
    return replan(*b);
}

alsub_status alsub_batch_refine(alsub_batch_t b, void *stream) {
    if (!b) return report(ALSUB_ERR_INVALID_ARG, "NULL batch");
    return run(*b, (cudaStream_t)stream);
}

alsub_status alsub_batch_tune(alsub_batch_t b, void *stream, int32_t *block, int32_t *blocks_per_sm,
                              float *best_ms) {
    if (!b) return report(ALSUB_ERR_INVALID_ARG, "NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks[] = {128, 256, 512};
    const int pers[] = {0, 2, 4, 8};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bb = b->block, bp = b->blocks_per_sm;
    for (int blk : blocks) {
        for (int p : pers) {
            b->block = blk;
            b->blocks_per_sm = p;
            alsub_status st = replan(*b);
            if (st) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
            for (int w = 0; w < 2; w++)
                if ((st = run(*b, s))) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
            cudaEventRecord(e0, s);
            for (int k = 0; k < 5; k++) run(*b, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 5.f;
            if (ms < best) { best = ms; bb = blk; bp = p; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->block = bb;
    b->blocks_per_sm = bp;
    alsub_status st = replan(*b);
    if (st) return st;
    if (block) *block = bb;
    if (blocks_per_sm) *blocks_per_sm = bp;
    if (best_ms) *best_ms = best;
    return ALSUB_OK;
}

alsub_status alsub_batch_launches(alsub_batch_t b, int64_t *launches) {
    if (!b || !launches) return report(ALSUB_ERR_INVALID_ARG, "bad arguments");
    *launches = b->launches;
    return ALSUB_OK;
}

alsub_status alsub_batch_destroy(alsub_batch_t b) {
    if (!b) return ALSUB_OK;
    cudaDeviceSynchronize();
    drop_graph(*b);
    free_plans(*b);
    delete b;
    return ALSUB_OK;
}

}  // extern "C"
