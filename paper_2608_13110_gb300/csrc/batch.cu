// Batched evaluation of many circuits of uneven size, recorded once into a
// CUDA graph and replayed with one launch (the paper's production mode runs
// many independent contractions of one topology, Sec. 5.2; here the circuits
// may differ in n and d).
//
// Layout of the caller's workspace: for every item, its plan's tables, then
// (wide items only) one rescaling/partial/boundary region per bitstring;
// then the array of narrow-item descriptors. Narrow items (width <= 12) run
// as one multi-item launch, one CTA per bitstring; wide items run the HBM
// pass sequence with all of their bitstrings side by side, spread over
// parallel graph branches by estimated cost (longest first onto the least
// loaded branch).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "misc_kernels.cuh"
#include "tb_plan.h"
#include "tb_run.h"
#include "tbsweep.h"

using namespace tb;
using namespace tb::rt;

struct tb_batch {
    std::vector<tb_batch_item> items;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nbranches = 0;
    int64_t narrow_blocks = 0;
};

namespace {

struct Layout {
    std::vector<int64_t> off;  // workspace offset of each item's tables
    std::vector<int64_t> len;  // bytes of each item's region
    int64_t items_off = 0;     // narrow descriptors
    int64_t total = 0;
    int n_narrow = 0;
};

bool layout_of(const tb_batch_item* items, int nitems, Layout& L, std::string& err) {
    L = Layout();
    int64_t off = 0;
    for (int i = 0; i < nitems; ++i) {
        const tb_batch_item& it = items[i];
        if (!it.plan || it.nb < 0 || (it.nb > 0 && (!it.d_bits || !it.d_out))) {
            err = "item " + std::to_string(i) + ": NULL plan, buffer or negative count";
            return false;
        }
        const Plan& P = it.plan->p;
        if (P.h > MAX_H) {
            err = "item " + std::to_string(i) + ": boundary wider than 2^33 entries";
            return false;
        }
        if (P.open_k) {
            err = "item " + std::to_string(i) + ": open plans are evaluated by tb_amplitudes / tb_amplitudes_device";
            return false;
        }
        const CallLayout c = call_layout(P);
        const int64_t len = align_up(P.lay.total, 256) + it.nb * c.per_b;
        L.off.push_back(off);
        L.len.push_back(len);
        off += len;
        if (small_path(P) && it.nb > 0) ++L.n_narrow;
    }
    L.items_off = off;
    off += align_up((int64_t)std::max(1, L.n_narrow) * (int64_t)sizeof(SmallItem), 256);
    L.total = off;
    return true;
}

template <class T>
const T* at(const void* ws, int64_t off) {
    return reinterpret_cast<const T*>(static_cast<const uint8_t*>(ws) + off);
}

}  // namespace

extern "C" {

int64_t tb_batch_workspace_bytes(const tb_batch_item* items, int nitems) {
    if (!items || nitems <= 0) return -1;
    Layout L;
    std::string err;
    if (!layout_of(items, nitems, L, err)) return -1;
    return L.total;
}

int tb_batch_create(const tb_batch_item* items, int nitems, void* d_ws, int64_t ws_bytes, int nbranches,
                    void* stream, tb_batch** out) {
    if (!out || !items || nitems <= 0 || !d_ws) return fail(TB_EINVAL, "NULL or empty argument");
    *out = nullptr;
    Layout L;
    std::string err;
    if (!layout_of(items, nitems, L, err)) return fail(TB_EINVAL, err);
    if (ws_bytes < L.total)
        return fail(TB_ENOMEM, "batch workspace needs " + std::to_string(L.total) + " bytes");
    nbranches = std::max(1, std::min(nbranches <= 0 ? 4 : nbranches, 16));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(d_ws);

    // tables of every item, and the narrow descriptors
    std::vector<SmallItem> narrow;
    int64_t nblocks = 0;
    int hmax = 1;
    for (int i = 0; i < nitems; ++i) {
        const Plan& P = items[i].plan->p;
        TB_CUDA(cudaMemcpyAsync(ws + L.off[i], P.blob.data(), (size_t)P.lay.total, cudaMemcpyHostToDevice, st));
        if (!small_path(P) || items[i].nb == 0) continue;
        const TableLayout& T = P.lay;
        const uint8_t* base = ws + L.off[i];
        SmallItem si;
        std::memset(&si, 0, sizeof(si));
        si.p.n = P.n;
        si.p.h = P.h;
        si.p.nb = (int)items[i].nb;
        si.p.bits = items[i].d_bits;
        si.p.steps = at<StepG>(base, T.steps);
        si.p.tgt = at<int8_t>(base, T.step_tgt);
        si.p.ctl = at<int8_t>(base, T.step_ctl);
        si.p.xq = at<int16_t>(base, T.step_xq);
        si.p.row_end = at<int32_t>(base, T.row_end);
        si.p.nrows = (int)P.row_end.size();
        si.p.init_low = at<float2>(base, T.init_low);
        si.p.init_top = at<float2>(base, T.init_top);
        si.p.red_low = at<float2>(base, T.red_low);
        si.p.out = items[i].d_out;
        si.first_block = nblocks;
        nblocks += items[i].nb;
        hmax = std::max(hmax, P.h);
        narrow.push_back(si);
    }
    if (!narrow.empty())
        TB_CUDA(cudaMemcpyAsync(ws + L.items_off, narrow.data(), narrow.size() * sizeof(SmallItem),
                                cudaMemcpyHostToDevice, st));
    TB_CUDA(cudaStreamSynchronize(st));

    // wide items onto branches, longest first onto the least loaded branch
    std::vector<int> wide;
    for (int i = 0; i < nitems; ++i)
        if (!small_path(items[i].plan->p) && items[i].nb > 0) wide.push_back(i);
    auto cost = [&](int i) {
        const Plan& P = items[i].plan->p;
        return (double)items[i].nb * (double)(P.n_pass_launches() + 2) * std::ldexp(1.0, P.h);
    };
    std::sort(wide.begin(), wide.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<std::vector<int>> branch(nbranches);
    std::vector<double> load(nbranches, 0.0);
    for (int i : wide) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        branch[k].push_back(i);
        load[k] += cost(i);
    }

    tb_batch* B = nullptr;
    try {
        B = new tb_batch;
    } catch (const std::bad_alloc&) {
        return fail(TB_ENOMEM, "host allocation failed");
    }
    B->items.assign(items, items + nitems);
    B->nbranches = nbranches;
    B->narrow_blocks = nblocks;

    // record: origin -> (narrow launch | branch 0..k-1) -> origin
    std::vector<cudaStream_t> ss(nbranches + 1, nullptr);
    std::vector<cudaEvent_t> ev(nbranches + 1, nullptr);
    int rc = TB_OK;
    auto cleanup = [&]() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        for (auto s : ss)
            if (s) cudaStreamDestroy(s);
    };
    for (int k = 0; k <= nbranches && rc == TB_OK; ++k) {
        if (cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess)
            rc = fail(TB_ECUDA, "stream or event creation failed");
    }
    if (rc == TB_OK) {
        cudaStream_t origin = ss[nbranches];
        cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = fail(TB_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
        if (rc == TB_OK) {
            cudaEventRecord(ev[nbranches], origin);
            if (!narrow.empty()) {
                e = launch_small_multi(at<SmallItem>(ws, L.items_off), (int)narrow.size(), nblocks, hmax, origin);
                if (e != cudaSuccess) rc = fail(TB_ECUDA, std::string("narrow launch: ") + cudaGetErrorString(e));
            }
            for (int k = 0; k < nbranches && rc == TB_OK; ++k) {
                cudaStreamWaitEvent(ss[k], ev[nbranches], 0);
                for (int i : branch[k]) {
                    const Plan& P = items[i].plan->p;
                    rc = run_device(P, items[i].d_bits, items[i].nb, ws + L.off[i], L.len[i],
                                    align_up(P.lay.total, 256), items[i].d_out, ss[k]);
                    if (rc != TB_OK) break;
                }
                cudaEventRecord(ev[k], ss[k]);
                cudaStreamWaitEvent(origin, ev[k], 0);
            }
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(origin, &g);
            if (rc == TB_OK && e != cudaSuccess)
                rc = fail(TB_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
            if (rc == TB_OK) {
                B->graph = g;
                e = cudaGraphInstantiate(&B->exec, g, 0);
                if (e != cudaSuccess) rc = fail(TB_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
    }
    cleanup();
    if (rc != TB_OK) {
        tb_batch_destroy(B);
        return rc;
    }
    *out = B;
    return TB_OK;
}

int tb_batch_launch(tb_batch* batch, void* stream) {
    if (!batch || !batch->exec) return fail(TB_EINVAL, "NULL batch");
    TB_CUDA(cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream)));
    return TB_OK;
}

void tb_batch_destroy(tb_batch* batch) {
    if (!batch) return;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    delete batch;
}

}  // extern "C"
