// Device-driven round loop: the peel rounds of Alg. 1 whose supports come from
// the decremental update, run back to back on the GPU without a host
// synchronisation per round.
//
// Alg. 1 repeats "supports, prune" until a round removes nothing; the host
// driver of capi.cu reads the round counters after every prune to decide what
// comes next.  Once the supports of a round come from the decremental update
// (update.cu), a round is a fixed sequence of kernels whose sizes are known
// only on the device: prune + tile scan, a decision, the update, the
// compaction.  This file captures that sequence once per handle into a CUDA
// graph,
//
//   WHILE (continue) { SWITCH (buffer of the current graph) { round 0->1 | round 1->0 } }
//
// where every kernel reads the live edge count, the threshold and the round's
// decision from a device control block (LoopCtl) and loops over its work with
// a fixed grid, the decide kernel writes one record per round, and the end
// kernel advances the control block and sets the loop condition.  The loop
// stops when a round removes nothing (fixed K: the host finalizes), when no
// edge is left, when the next supports need a support step (the update rule
// chose to recompute), or when its record capacity is reached; the host then
// reads the control block and the records once.
//
// The K sweep (ktruss_decompose) runs in the same loop: a round that removes
// nothing raises K and copies the graph into the other buffer with its
// supports, so that the two cases of the switch always alternate buffers.
#include <cuda_runtime.h>

#include "ktruss.h"
#include "ktruss_internal.cuh"

namespace kt {
namespace {

// The update rule of the host driver (capi.cu, use_update), on the device.
__device__ __forceinline__ bool use_update_dev(int32_t mode, int32_t removed_tri, int32_t kept) {
    if (mode == KTRUSS_UPDATE_NEVER || kept == 0) return false;
    if (mode == KTRUSS_UPDATE_ALWAYS) return true;
    return int64_t(removed_tri) * 4 <= int64_t(kept);
}

__global__ void loop_switch_kernel(const LoopCtl *lc, cudaGraphConditionalHandle hs) {
    cudaGraphSetConditional(hs, unsigned(lc->buf));
}

// After prune + tile scan: the round's record and decision.
__global__ void loop_decide_kernel(LoopCtl *lc, RoundCounters *cnt, LoopRecord *rec) {
    const int32_t m = lc->m, kept = cnt[0].kept, listed = cnt[0].removed_tri;
    const int32_t removed = m - kept;
    if (!lc->decompose || lc->fresh) {
        // a new live graph: its triangles are those of the previous one minus
        // the ones the update destroyed
        if (lc->updated) lc->tri -= (long long)cnt[1].triangles;
        LoopRecord r;
        r.live = m;
        r.removed = removed;
        r.upd = lc->updated;
        r.pad = 0;
        r.tri = lc->tri;
        rec[lc->rec++] = r;
    } else {
        rec[lc->rec - 1].removed += removed;  // same graph at a higher K
    }
    cnt[1].triangles = 0;
    lc->fresh = 0;
    int32_t a = 0;
    if (removed == 0) {
        // fixed K: converged.  K sweep: the graph is the K-truss; the next K
        // starts from it with the same supports, copied to the other buffer
        if (lc->decompose) {
            lc->thr += 1;
            a = kActCompact | kActCarry;
        }
    } else {
        const bool upd = use_update_dev(lc->update_mode, listed, kept);
        a = kActCompact | (upd ? (kActUpdate | kActCarry) : 0);
        lc->nlist = listed;
        lc->level = lc->thr + 1;  // trussness of the edges the K-truss loses
        lc->fresh = 1;
        lc->updated = upd ? 1 : 0;
    }
    lc->action = a;
}

// After the compaction: advance to the next graph and set the loop condition.
__global__ void loop_end_kernel(LoopCtl *lc, RoundCounters *cnt, cudaGraphConditionalHandle hw) {
    const int32_t a = lc->action;
    bool cont = false;
    if (a & kActCompact) {
        lc->m = cnt[0].kept;
        lc->buf ^= 1;
        if (lc->m == 0) {
            lc->status = kLoopEmpty;
        } else if (!(a & kActCarry)) {
            lc->status = kLoopNeedSupport;
        } else {
            lc->status = kLoopRunning;
            cont = true;
        }
    } else {
        lc->status = kLoopConverged;
    }
    lc->iters += 1;
    if (cont && (lc->rec >= lc->rec_cap || lc->iters >= lc->iter_cap)) {
        cont = false;
        lc->status = kLoopCap;
    }
    cnt[0].removed_tri = 0;
    cudaGraphSetConditional(hw, cont ? 1u : 0u);
}

// One round reading buffer p and writing buffer p ^ 1, captured on stream s.
cudaError_t capture_round(const LoopBuffers &b, int p, cudaGraphConditionalHandle hw,
                          cudaStream_t s) {
    int launches = 0;
    const int q = p ^ 1;
    const Live cur{b.rp[p], b.col[p], b.eid[p], b.n, b.cap_m};
    UpdateState ust = *b.ust;
    ust.ldeg_valid = true;  // the loop starts with current lower degrees
    cudaError_t e = launch_prune_count(b.S[p], b.cap_m, 0, b.tile_count, b.tile_off, b.cnt, s,
                                       &launches, b.keep, b.us.list, b.col[p], ust.ldeg, b.lc);
    if (e != cudaSuccess) return e;
    loop_decide_kernel<<<1, 1, 0, s>>>(b.lc, b.cnt, b.rec);
    e = launch_support_update(cur, b.keep, b.us.list, b.cap_m, b.S[p], &b.cnt[1].triangles, b.us,
                              &ust, s, &launches, nullptr, nullptr, nullptr, b.lc);
    if (e != cudaSuccess) return e;
    e = launch_compact(cur, b.S[p], 0, b.tile_off, b.cnt, b.pos, b.rp[q], b.col[q], b.eid[q],
                       nullptr, nullptr, s, &launches, nullptr, 0, b.keep, b.S[q], b.lc);
    if (e != cudaSuccess) return e;
    loop_end_kernel<<<1, 1, 0, s>>>(b.lc, b.cnt, hw);
    return cudaGetLastError();
}

}  // namespace

cudaError_t loop_graph_build(LoopGraph *lg, const LoopBuffers &b) {
    if (lg->exec) return cudaSuccess;
    cudaStream_t s = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle hw = 0, hs = 0;
    cudaGraphNode_t wnode = nullptr, knode = nullptr, snode = nullptr;
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = hw;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
        if (e == cudaSuccess) body = wp.conditional.phGraph_out[0];
    }
    // body: the switch value from the control block, then the switch
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hs, body, 0, 0);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        loop_switch_kernel<<<1, 1, 0, s>>>(b.lc, hs);
        cudaError_t le = cudaGetLastError();
        e = cudaStreamEndCapture(s, &body);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) {
        size_t count = 1;
        e = cudaGraphGetNodes(body, &knode, &count);
        if (e == cudaSuccess && count != 1) e = cudaErrorInvalidValue;
    }
    cudaGraph_t cases[2] = {nullptr, nullptr};
    if (e == cudaSuccess) {
        cudaGraphNodeParams sp = {};
        sp.type = cudaGraphNodeTypeConditional;
        sp.conditional.handle = hs;
        sp.conditional.type = cudaGraphCondTypeSwitch;
        sp.conditional.size = 2;
        e = cudaGraphAddNode(&snode, body, &knode, nullptr, 1, &sp);
        if (e == cudaSuccess) {
            cases[0] = sp.conditional.phGraph_out[0];
            cases[1] = sp.conditional.phGraph_out[1];
        }
    }
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        e = cudaStreamBeginCaptureToGraph(s, cases[p], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t ce = capture_round(b, p, hw, s);
        e = cudaStreamEndCapture(s, &cases[p]);
        if (e == cudaSuccess) e = ce;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGetLastError();
        return e;
    }
    lg->exec = exec;
    return cudaSuccess;
}

void loop_graph_destroy(LoopGraph *lg) {
    if (lg->exec) cudaGraphExecDestroy(lg->exec);
    lg->exec = nullptr;
}

}  // namespace kt
