// blocked_launch.cuh -- workspace planning and the host sweep loop of the
// multi-kernel path, instantiated once per scalar type by blocked_{s,d,c,z}.cu.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "blocked_layout.h"
#include "gesvj_blocked.cuh"
#include "gesvj_pairstep.cuh"
#include "launch_util.cuh"
#include "internal.h"

namespace bsvd {

// End of a sweep inside the device-side sweep loop: count the sweep and keep
// looping while some matrix is still active and fewer than max_sweeps sweeps
// have run.  The count starts at zero each launch (the host clears it), and
// a negative value is read as zero, so the loop ends after at most
// max_sweeps sweeps whatever the counter held.
static __global__ void blk_continue(cudaGraphConditionalHandle h, const BlockedArgs a) {
    int* counter = a.any_active + 1;
    const int c = max(*counter, 0) + 1;
    *counter = c;
    cudaGraphSetConditional(h, (*a.any_active != 0 && c < a.max_sweeps) ? 1u : 0u);
}

// The masked sweep loop as one CUDA graph: a conditional WHILE node whose
// body is one sweep (every round's launches, the convergence kernel) plus
// blk_continue, which stops the loop on the device once no matrix is
// active.  No sweep is issued after the batch has converged and the host
// never waits.  Returns cudaErrorNotSupported, having queued nothing, when
// the graph cannot be built (the caller then replays a plain one-sweep
// graph max_sweeps times).
template <class Sweep>
cudaError_t blk_run_while(const BlockedArgs& a, cudaStream_t st, cudaStream_t capture, Sweep& sweep) {
    if (a.max_sweeps < 1) return cudaErrorNotSupported;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t node;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = ok && cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
    if (ok) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
            cudaSuccess) {
            cudaError_t ce = sweep(capture);
            if (ce == cudaSuccess) {
                blk_continue<<<1, 1, 0, capture>>>(h, a);
                ce = cudaGetLastError();
            }
            cudaGraph_t out = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(capture, &out);
            ok = ce == cudaSuccess && ee == cudaSuccess && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
        } else {
            ok = false;
        }
    }
    cudaError_t e = cudaErrorNotSupported;
    if (ok) {
        e = cudaMemsetAsync(a.any_active + 1, 0, sizeof(int), st);   // the sweep counter
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    } else {
        cudaGetLastError();
    }
    if (exec) cudaGraphExecDestroy(exec);   // freed once the queued launch finishes
    if (g) cudaGraphDestroy(g);
    return e;
}

template <int NB> struct BlkCfg;
template <> struct BlkCfg<4>  { static constexpr int GT = 32; };
template <> struct BlkCfg<8>  { static constexpr int GT = 64; };
template <> struct BlkCfg<16> { static constexpr int GT = 128; };
template <> struct BlkCfg<32> { static constexpr int GT = 256; };

// `var` (nullptr for a batch of one shape) gives a variable-shape batch: each
// matrix's shape and workspace offsets, and the maxima that size the grids;
// a smaller matrix's CTAs return at once in the rounds, pairs and rows it
// does not have.
template <class T, int NB>
cudaError_t blk_run_nb(BlockedArgs a, void* work, cudaStream_t st, bool two_stage, bool host_sync,
                       cudaStream_t capture, const BlkVarPlan* var) {
    using R = Real<T>;
    constexpr int TWO = 2 * NB, GT = BlkCfg<NB>::GT, LDG = TWO + 1;
    cudaError_t e;
    long long nW, nV, nG, nJ;                  // region sizes, elements
    if (!var) {
        const BlkSizes z = blk_sizes(NB, a.M, a.N, two_stage);
        a.l = z.l; a.L = z.L; a.Np = z.Np;
        a.sW = z.W; a.sVw = z.V; a.sG = z.G; a.sJ = z.J; a.sT = z.T;
        nW = a.count * z.W; nV = a.count * z.V; nG = a.count * z.G; nJ = a.count * z.J;
        a.shapes = nullptr;
    } else {
        if (two_stage || (int)var->shapes.size() != a.count) return cudaErrorInvalidValue;
        a.M = var->Mmax; a.N = var->Nmax; a.l = var->lmax; a.L = var->Lmax; a.Np = var->lmax * NB;
        a.sW = a.sVw = a.sG = a.sJ = a.sT = 0;
        nW = var->W; nV = var->V; nG = var->G; nJ = var->J;
    }
    char* p = static_cast<char*>(work);
    a.state = reinterpret_cast<int*>(p);       p += blk_align((size_t)a.count * 4 * sizeof(int));
    a.pairflag = reinterpret_cast<int*>(p);    p += blk_align((size_t)a.count * (a.L / 2) * sizeof(int));
    a.any_active = reinterpret_cast<int*>(p);  p += blk_align(sizeof(int));
    if (var) {
        BlkShape* sh = reinterpret_cast<BlkShape*>(p);
        p += blk_align((size_t)a.count * sizeof(BlkShape));
        // pageable source: the call returns once the records are staged
        if ((e = cudaMemcpyAsync(sh, var->shapes.data(), (size_t)a.count * sizeof(BlkShape),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return e;
        a.shapes = sh;
    }
    T* base = reinterpret_cast<T*>(p);
    a.W = base;  base += (size_t)nW;
    a.Vw = base; base += (size_t)nV;
    a.G = base;  base += (size_t)nG;
    a.J = base;  base += (size_t)nJ;
    a.T = base;

    const int heevj_smem = 2 * TWO * LDG * (int)sizeof(T) + InnerTables<T, NB>::bytes();
    const int fin_smem = (kBlkThreads / 32) * (int)sizeof(R) + 16 + 2 * (int)sizeof(T) +
                         a.N * ((int)sizeof(R) + 4) + 16;
    // J, column stride up to 2nb + 1; real FP32 J's split-TF32 fragments
    const int upd_smem = std::max(TWO * (TWO + 1) * (int)sizeof(T),
                                  std::is_same<T, float>::value    ? j_fragment_bytes<NB>()
                                  : std::is_same<T, float2>::value ? jc_fragment_bytes<NB>() : 0);
    if ((e = allow_dynamic_smem<blk_heevj<T, NB, GT>>()) != cudaSuccess ||
        (e = allow_dynamic_smem<blk_finalize<T>>()) != cudaSuccess ||
        (e = allow_dynamic_smem<blk_update_fused<T, NB>>()) != cudaSuccess ||
        (e = allow_dynamic_smem<blk_update_stage1<T, NB>>()) != cudaSuccess ||
        (e = allow_dynamic_smem<blk_update_stage2<T, NB>>()) != cudaSuccess)
        return e;
    // single precision, nb = 8 or 16, tensor cores: one pair-step kernel per
    // round (flags bit 12: the three kernels)
    constexpr bool kPairCapable = (std::is_same<T, float>::value || std::is_same<T, float2>::value) && (NB == 8 || NB == 16);
    const bool pairstep = kPairCapable && !two_stage && !(a.flags & (128 | 4096));
    if constexpr (kPairCapable)
        if (pairstep && (e = allow_dynamic_smem<blk_pairstep<T, NB>>()) != cudaSuccess) return e;

    blk_load<T><<<a.count, kBlkThreads, 0, st>>>(a);
    const dim3 gpair(a.count, a.L / 2);
    // row blocks of the update: all of them, unless the block pairs alone
    // give more than about 16 CTAs per SM (then each CTA loops over several;
    // the two-stage kernels take one row block per CTA)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    const long long pairs = (long long)a.count * (a.L / 2);
    const int zrows = (a.M + a.N + kUpdRows - 1) / kUpdRows;
    const int zcap = (int)std::max(1LL, (16LL * sms + pairs - 1) / pairs);
    const dim3 gupd(a.count, a.L / 2, two_stage ? zrows : std::min(zrows, zcap));
    // one sweep: every round's stages, then the end-of-sweep bookkeeping
    auto sweep = [&](cudaStream_t s) -> cudaError_t {
        for (int r = 0; r < a.L - 1; ++r) {
            if constexpr (kPairCapable)
                if (pairstep) {
                    blk_pairstep<T, NB><<<gpair, kPairThreads, PairLayout<T, NB>::kBytes, s>>>(a, r);
                    continue;
                }
            // real FP32: the tensor cores (flags bit 7: FMA register tiles)
            if constexpr (std::is_same<T, float>::value && (NB == 8 || NB == 16)) {
                if (a.flags & 128) blk_gram_f32<NB><<<gpair, kBlkThreads, 0, s>>>(a, r);
                else blk_gram_f32_tc<NB><<<gpair, kBlkThreads, 0, s>>>(a, r);
            } else if constexpr (std::is_same<T, float>::value && NB >= 8) {
                blk_gram_f32<NB><<<gpair, kBlkThreads, 0, s>>>(a, r);
            } else if constexpr (std::is_same<T, float2>::value && (NB == 8 || NB == 16)) {
                // complex64: the tensor cores (flags bit 7: the FMA pipes)
                if (a.flags & 128) blk_gram<T, NB><<<gpair, kBlkThreads, 0, s>>>(a, r);
                else blk_gram_c64_tc<NB><<<gpair, kBlkThreads, 0, s>>>(a, r);
            }
            else
                blk_gram<T, NB><<<gpair, kBlkThreads, 0, s>>>(a, r);
            blk_heevj<T, NB, GT><<<gpair, GT, heevj_smem, s>>>(a, r);
            if (two_stage) {
                blk_update_stage1<T, NB><<<gupd, kUpdRows, upd_smem, s>>>(a, r);
                blk_update_stage2<T, NB><<<gupd, kUpdRows, upd_smem, s>>>(a, r);
            } else {
                blk_update_fused<T, NB><<<gupd, kUpdRows, upd_smem, s>>>(a, r);
            }
        }
        cudaError_t err = cudaMemsetAsync(a.any_active, 0, sizeof(int), s);
        if (err != cudaSuccess) return err;
        blk_converge<<<(a.count + 127) / 128, 128, 0, s>>>(a);
        return cudaGetLastError();
    };
    if (host_sync) {
        // batch-level convergence (the paper's unmasked design): stop once no
        // matrix rotated in the last sweep
        for (int sw = 0; sw < a.max_sweeps; ++sw) {
            if ((e = sweep(st)) != cudaSuccess) return e;
            int any = 0;
            if ((e = cudaMemcpyAsync(&any, a.any_active, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            if (!any) break;
        }
    } else if (capture && !(a.flags & 2048) && (e = blk_run_while(a, st, capture, sweep)) != cudaErrorNotSupported) {
        // the sweep loop ran (or failed) as one graph with a device-side loop
        if (e != cudaSuccess) return e;
    } else {
        // masked: converged matrices skip every stage, so max_sweeps sweeps are
        // issued without a host round trip; one sweep is recorded once into a
        // CUDA graph (on the private capture stream) and replayed per sweep
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool graphed = false;
        if (capture && cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t ce = sweep(capture);
            const cudaError_t ee = cudaStreamEndCapture(capture, &graph);
            graphed = ce == cudaSuccess && ee == cudaSuccess && graph &&
                      cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (!graphed) cudaGetLastError();
        }
        // flags bit 4: every kSyncEvery sweeps read the batch's any-active flag
        // on the host and stop launching once every matrix has converged
        constexpr int kSyncEvery = 4;
        for (int sw = 0; sw < a.max_sweeps; ++sw) {
            e = graphed ? cudaGraphLaunch(exec, st) : sweep(st);
            if (e != cudaSuccess) break;
            if ((a.flags & 16) && sw % kSyncEvery == kSyncEvery - 1 && sw + 1 < a.max_sweeps) {
                int any = 0;
                if ((e = cudaMemcpyAsync(&any, a.any_active, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(st)) != cudaSuccess)
                    break;
                if (!any) break;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);   // freed once the queued launches finish
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return e;
    }
    blk_finalize<T><<<a.count, kBlkThreads, fin_smem, st>>>(a);
    if (a.trans ? a.wantU : a.wantV) {
        const int nt = (a.N + kFinBT - 1) / kFinBT;
        const dim3 gfin(a.count, nt, nt);
        if (!(a.flags & 1)) blk_fin_gram<T><<<gfin, kFinThreads, 0, st>>>(a);
        blk_fin_z<T><<<gfin, kFinThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t blk_run(int nb, const BlockedArgs& a, void* work, cudaStream_t st, bool two_stage, bool host_sync,
                    cudaStream_t capture, const BlkVarPlan* var = nullptr) {
    switch (nb) {
        case 4: return blk_run_nb<T, 4>(a, work, st, two_stage, host_sync, capture, var);
        case 8: return blk_run_nb<T, 8>(a, work, st, two_stage, host_sync, capture, var);
        case 16: return blk_run_nb<T, 16>(a, work, st, two_stage, host_sync, capture, var);
        case 32: return blk_run_nb<T, 32>(a, work, st, two_stage, host_sync, capture, var);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsvd

#define BSVD_DEFINE_BLOCKED(TYPE, TAG)                                                          \
    cudaError_t bsvd::blocked_run_##TAG(int nb, const BlockedArgs& a, void* work, cudaStream_t st, \
                                        bool two_stage, bool host_sync, cudaStream_t capture) { \
        return blk_run<TYPE>(nb, a, work, st, two_stage, host_sync, capture);                   \
    }                                                                                           \
    cudaError_t bsvd::blocked_run_var_##TAG(int nb, const BlockedArgs& a, const BlkVarPlan& var, \
                                            void* work, cudaStream_t st, cudaStream_t capture) {  \
        return blk_run<TYPE>(nb, a, work, st, false, false, capture, &var);                     \
    }
