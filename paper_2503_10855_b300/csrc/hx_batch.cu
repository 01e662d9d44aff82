// hx_batch.cu -- many independent nest instances in one persistent launch.
//
// The Hercules host backend runs independent calls and the iterations of
// parallel fork-joins as concurrent tasks (Sec. 4.5; the AsyncCall attribute
// of Sec. 3.4).  On one GPU that becomes a device work-list: every instance
// is cut into the same tiles its standalone call would use, the tiles of all
// instances are described once and resident workers take their work items.
// Map->reduce tiles and stencil blocks form WARP runs (a warp computes and
// reduces a run of consecutive tiles of one instance on its own, with no
// block barrier); histogram chunks are CTA items (the CTA's warps share one
// set of shared-memory counters) and run first.  Work items only store their
// partial results (map tile partials; atomic max / add into the instance's
// accumulator for stencils and histograms): no fences, no arrival tickets.
// A second launch, chained with programmatic dependent launch, runs the
// final combine of every instance the launch completed, one CTA each.  A
// stencil instance with several sweeps runs all of them in the same launch:
// the runs of its sweep s wait (bounded) for its sweep s - 1; no other work
// item ever waits.  The older schedule -- one launch per sweep ("rounds") --
// remains available for comparison.
#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <string>
#include <new>
#include <vector>

#include "hx_batch.cuh"

namespace hx {

// One histogram chunk counted by the whole CTA into its shared counters
// (dynamic shared memory, kHiSmemBytes) and added into the instance's bins.
// Each thread keeps kBHiDepth 16-byte loads in flight.
constexpr int kBHiDepth = 8;
__device__ __forceinline__ void batch_hist_item(const BInst &I, int64_t tile, unsigned int *sh) {
    hist_zero(sh);
    __syncthreads();
    const unsigned int slot = hist_slot_offset();
    const uint8_t *v = static_cast<const uint8_t *>(I.in0);
    const int64_t s = tile * kBHiTile;
    const int64_t e = min(I.n, s + kBHiTile);
    int head = (int)((16 - ((uintptr_t)(v + s) & 15u)) & 15u);
    if (head > e - s) head = (int)(e - s);
    const int64_t nvec = (e - s - head) / 16;
    const int tail = (int)((e - s - head) % 16);
    hist_count_strided<kBHiDepth>(sh, slot, reinterpret_cast<const uint4 *>(v + s + head), threadIdx.x,
                                  kBatchThreads, nvec);
    if (threadIdx.x < head) hist_count_byte(sh, slot, v[s + threadIdx.x]);
    if (threadIdx.x < tail) hist_count_byte(sh, slot, v[e - tail + threadIdx.x]);
    __syncthreads();
    hist_merge(sh, I.acc);
    __syncthreads();
}

// L2 prefetch of the rows of a stencil warp block that the previous block of
// its run did not load, rows r_begin + 1 .. r_begin + R (clamped): each lane
// the line of its first column.  Issued one block ahead, it keeps a second
// block's DRAM requests in flight without holding registers, and the block's
// own loads then find their rows in L2.  (Prefetching the halo columns too,
// or one bulk prefetch per row, measured slower.)  A prefetch only moves
// lines into L2, the point of coherence, so it is safe for grids that the
// launch writes, and it changes no result.
template <int R>
__device__ __forceinline__ void prefetch_stencil_block(const float *src, int nx, int ny, int c_begin, int r_begin,
                                                       int lane) {
    const int c0 = c_begin + lane * 4;
    if (c0 >= nx) return;
#pragma unroll
    for (int k = 1; k <= R; ++k) {
        const int r = r_begin + k < ny ? r_begin + k : ny - 1;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(src + (size_t)r * nx + c0));
    }
}

// Index i of the instance with prefix[i] <= j < prefix[i + 1] (instances
// with no items have equal neighbours and are never returned).
__device__ __forceinline__ unsigned int find_instance(const uint32_t *__restrict__ prefix, unsigned int n_inst,
                                                      unsigned int j) {
    unsigned int lo = 0, hi = n_inst;
    while (hi - lo > 1) {
        const unsigned int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until the blocks a run of sweep `phase` depends on have finished
// sweep phase - 1.  The run is blocks first .. first + cnt - 1 (block t is
// column t / tiles_y, row t % tiles_y; consecutive blocks go down a column),
// so its dependencies are each block itself and its west and east
// neighbours, plus the north neighbour of the first block and the south
// neighbour of the last (the other north / south neighbours are blocks of
// the run).  Lane 3k + j checks block k itself (j = 0), west (1) or east (2);
// lanes 3 cnt and 3 cnt + 1 the north and south ends: one progress word per
// lane, so a satisfied wait costs one round trip.  A lane polls its word with
// ld.acquire, exponential back-off (32 ns .. 1 us) and a deadline of
// sync.limit_ns; on running out it records HX_ERR_TIMEOUT and gives up.  The
// warp barrier then orders every lane's grid reads after the acquires.
__device__ __forceinline__ void wait_blocks(const BInst &I, int64_t first, unsigned int cnt, int phase,
                                            const BatchSync &sync, int lane) {
    const int64_t ty = I.tiles_y, last = first + cnt - 1;
    int64_t dep = -1;
    if (lane < 3 * (int)cnt) {
        const int64_t t = first + lane / 3;
        const int j = lane % 3;
        dep = j == 0 ? t : (j == 1 ? (t >= ty ? t - ty : -1) : (t + ty < I.tiles ? t + ty : -1));
    } else if (lane == 3 * (int)cnt) {
        dep = first % ty > 0 ? first - 1 : -1;
    } else if (lane == 3 * (int)cnt + 1) {
        dep = last % ty + 1 < ty ? last + 1 : -1;
    }
    const unsigned int need = (unsigned int)phase + (I.stall ? (1u << 20) : 0u);
    if (dep >= 0 && ld_acquire_u32(I.done + dep) < need) {
        const unsigned long long t0 = globaltimer_ns();
        unsigned int nap = 32;
        while (ld_acquire_u32(I.done + dep) < need) {
            if (globaltimer_ns() - t0 > (unsigned long long)sync.limit_ns) {
                // host-mapped word: a plain store (no atomic over the host link)
                *reinterpret_cast<volatile unsigned int *>(sync.err) = (unsigned int)HX_ERR_TIMEOUT;
                break;
            }
            __nanosleep(nap);
            nap = min(2 * nap, 1024u);
        }
    }
    __syncwarp();
}

// Phase 1 runs the CTA items (histogram chunks, CTA c takes items c, c + G,
// ...); phase 2 the warp runs, fetched one at a time from a counter (each
// warp prefetches its next index while it works, and runs are large, so the
// counter sees a few thousand atomics per launch).  The work list is not
// stored: item j belongs to the pair whose prefix range holds j (binary
// search), and its tiles follow from the instance's slice and run length, so
// the host only uploads one descriptor per instance (and, with MULTI, one
// word per (instance, sweep) pair).
//
// MULTI: stencil instances may run several sweeps in this launch (the
// sequential outer loop of Sec. 4.4 rule 1, kept inside one persistent
// launch).  Runs are taken in pair order, in which an instance's sweep s - 1
// comes before its sweep s, so a run waits only for runs taken before it:
// the oldest unfinished run is always being processed and never waits, and
// every wait ends.  After computing its blocks a run publishes each block's
// progress (a release store of the sweeps done); a run of sweep s waits until
// its blocks and their four neighbours have finished sweep s - 1 (bounded,
// see BatchSync) and reads the grid through L2.  Sweeps of an instance
// therefore overlap as a wavefront instead of meeting at a barrier.  Grids,
// residuals and results are the same as the standalone calls': every block
// computes the same values from the same inputs, and a maximum does not
// depend on order.
template <bool MULTI>
__global__ void __launch_bounds__(kBatchThreads, 2)
batch_kernel(const BInst *__restrict__ insts, unsigned int n_inst, const uint32_t *__restrict__ cta_prefix,
             const uint32_t *__restrict__ run_prefix, const uint32_t *__restrict__ pairs, unsigned int n_pairs,
             int round, unsigned int *ctrl, BatchSync sync) {
    // No early launch_dependents: the final-combine kernel is launched as
    // the CTAs exit, so its CTAs do not wait on SM slots through the tail
    // (slots that kernels of concurrent streams can use meanwhile).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(16) unsigned int sh[];   // kHiSmemBytes when the round has CTA items
    const int lane = threadIdx.x & 31;
    const unsigned int n_cta = __ldg(cta_prefix + n_inst), n_runs = __ldg(run_prefix + n_pairs);

    for (unsigned int it = blockIdx.x; it < n_cta; it += gridDim.x) {
        const unsigned int i = find_instance(cta_prefix, n_inst, it);
        if (!HX_CHECK(i < n_inst, kChkBatchInst, i, n_inst)) continue;
        const BInst &I = insts[i];
        batch_hist_item(I, I.t_first + (it - __ldg(cta_prefix + i)), sh);
    }

    // Warp runs are taken dynamically: lane 0 fetches the next run index
    // from ctrl[0] while the current run is processed (runs differ in cost,
    // a static assignment leaves warps idle at the end).
    unsigned int it = 0u;
    if (lane == 0) it = atomicAdd(&ctrl[0], 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    while (it < n_runs) {
        unsigned int next = 0u;
        if (lane == 0) next = atomicAdd(&ctrl[0], 1u);
        const unsigned int kp = find_instance(run_prefix, n_pairs, it);
        const uint32_t pr = MULTI ? __ldg(pairs + kp) : kp;
        const unsigned int i = pr & (kMaxPairInstances - 1u);
        const int phase = MULTI ? (int)(pr >> 24) : 0;
        if (!HX_CHECK(kp < n_pairs && i < n_inst, kChkBatchInst, i, n_inst)) {
            it = __shfl_sync(0xffffffffu, next, 0);
            continue;
        }
        const BInst &I = insts[i];
        const int64_t first = I.t_first + (int64_t)(it - __ldg(run_prefix + kp)) * I.run_len;
        const unsigned int cnt = (unsigned int)min((int64_t)I.run_len, I.t_first + I.t_count - first);
        if (!HX_CHECK(first >= 0 && first + cnt <= I.tiles, kChkBatchRun, first + cnt, I.tiles)) {
            it = __shfl_sync(0xffffffffu, next, 0);
            continue;
        }
        if (I.kind == kKindMap) {
            const float *x = static_cast<const float *>(I.in0);
            const float *y = static_cast<const float *>(I.in1);
            float *out = static_cast<float *>(I.o0);
            for (int64_t k = 0; k < cnt; ++k) {
                const int64_t tile = first + k;
                // the run's next tile, when it is full, is prefetched as well
                const int V = I.plan.vecs_per_thread;
                const int pf = k + 1 < cnt && (tile + 2) * I.plan.tile_elems <= I.plan.n ? 2 * V : V;
                const ff part = mr_tile<2, 2>(x, y, out, I.a, I.plan, tile, I.vec != 0, lane, pf);
                if (lane == 0) st_keep2(I.partials + tile, make_float2(part.hi, part.lo));
            }
        } else {
            const int sweep = I.sweep0 + round + phase;
            const bool multi = MULTI && I.n_sweeps > 1;
            if (multi && phase > 0) wait_blocks(I, first, cnt, phase, sync, lane);
            const float *src = static_cast<const float *>((sweep & 1) ? I.in1 : I.in0);
            float *dst = const_cast<float *>(static_cast<const float *>((sweep & 1) ? I.in0 : I.in1));
            float m = 0.0f;
            for (unsigned int k = 0; k < cnt; ++k) {
                const unsigned int tile = (unsigned int)(first + k);
                const int wy = (int)(tile % (unsigned int)I.tiles_y), wx = (int)(tile / (unsigned int)I.tiles_y);
                const int c_begin = wx * 128, r_begin = wy * kBatchStRows;
                if (!HX_CHECK(c_begin < I.nx && r_begin < I.ny, kChkBatchStencil, c_begin, r_begin)) continue;
                if (k + 1 < cnt) {   // the run's next block, one block ahead
                    const unsigned int t1 = tile + 1u;
                    const int wy1 = (int)(t1 % (unsigned int)I.tiles_y), wx1 = (int)(t1 / (unsigned int)I.tiles_y);
                    prefetch_stencil_block<kBatchStRows>(src, I.nx, I.ny, wx1 * 128, wy1 * kBatchStRows, lane);
                }
                if constexpr (MULTI)
                    m = fmaxf(m, I.vec ? stencil_block_vec<kBatchStRows, true>(src, dst, I.nx, I.ny, c_begin, r_begin)
                                       : stencil_block_strided<kBatchStRows>(src, dst, I.nx, I.ny, c_begin, r_begin));
                else
                    m = fmaxf(m, I.vec ? stencil_block_vec<kBatchStRows>(src, dst, I.nx, I.ny, c_begin, r_begin)
                                       : stencil_block_scalar<kBatchStRows>(src, dst, I.nx, I.ny, c_begin, r_begin));
            }
            m = warp_max(m);
            if (lane == 0) atomicMax(I.acc + phase, __float_as_uint(m));
            if (multi && phase + 1 < I.n_sweeps) {
                // publish this run's blocks to the next sweep's readers:
                // release stores after the warp's barrier (no fence stall)
                __syncwarp();
                if (lane < (int)cnt) st_release_u32(I.done + first + lane, (unsigned int)(phase + 1));
            }
        }
        it = __shfl_sync(0xffffffffu, next, 0);
    }
}

// The final combine of every instance this launch completed (it had work
// items in the launch and its slice reached its last tile), one CTA per
// instance, after the batched kernel has finished (programmatic dependent
// launch waits for the whole grid): the sum of a map->reduce instance from
// its tile partials in the standalone call's fixed order (all 256 threads
// fold, one virtual lane each), the residual of each stencil sweep the launch
// ran, the bins and scan of a histogram (one warp).  Accumulators and block
// progress words are left at zero for the next use; the run counter is reset
// for the next launch.  Whether an instance had work: its CTA chunks, plus,
// in a launch without a pair list, entries i and i + 1 of the run prefix; a
// launch with a pair list (run_prefix NULL here) runs every instance's whole
// slice.
//
// The descriptors and prefixes are written only by host copies, never by a
// kernel: the plan's synchronous copies, or a server step's upload on the
// stream ahead of the batched kernel, which cannot start before that copy
// has completed (and this kernel starts only as the batched kernel's CTAs
// exit).  So each CTA reads its instance's descriptor (into shared memory)
// and work count before waiting for the batched grid: only the loads of what
// the grid wrote (partials, accumulators) remain on the path after it.
__global__ void __launch_bounds__(kBatchThreads)
batch_final_kernel(const BInst *__restrict__ insts, unsigned int n_inst, const uint32_t *__restrict__ cta_prefix,
                   const uint32_t *__restrict__ run_prefix, int round, unsigned int *ctrl) {
    __shared__ ff red[kMrFoldLanes];
    __shared__ BInst sI;
    __shared__ unsigned int s_work;
    static_assert(sizeof(BInst) % 8 == 0 && sizeof(BInst) / 8 <= kBatchThreads, "descriptor copy");
    const int lane = threadIdx.x & 31;
    const unsigned int i = blockIdx.x;   // one CTA per instance
    if (i < n_inst) {
        if (threadIdx.x < sizeof(BInst) / 8)
            reinterpret_cast<unsigned long long *>(&sI)[threadIdx.x] =
                __ldg(reinterpret_cast<const unsigned long long *>(insts + i) + threadIdx.x);
        // whether the instance had work in this launch: its CTA chunks and
        // its first-pass runs (a pair-ordered launch, run_prefix NULL, gives
        // every instance its whole slice; that case reads sI below)
        if (threadIdx.x == 0)
            s_work = (__ldg(cta_prefix + i + 1) - __ldg(cta_prefix + i)) +
                     (run_prefix ? __ldg(run_prefix + i + 1) - __ldg(run_prefix + i) : 0u);
    }
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl[0] = 0u;
    if (i >= n_inst) return;
    const BInst &I = sI;
    const unsigned int work = s_work + (run_prefix ? 0u : (I.t_count > 0 && I.kind != kKindHist ? 1u : 0u));
    if (work == 0 || I.t_first + I.t_count != I.tiles) return;
    if (I.kind == kKindStencil && I.n_sweeps > 1)   // progress words back to zero
        for (int64_t k = threadIdx.x; k < I.tiles; k += blockDim.x) I.done[k] = 0u;
    if (I.kind == kKindMap) {
        const ff sf = mr_final_cta(I.partials, I.plan.tiles, red);
        if (threadIdx.x == 0) {
            const double s = ff_to_double(sf);
            *static_cast<float *>(I.o1) = (float)s;
            if (I.o2) *static_cast<double *>(I.o2) = s;
        }
    } else if (threadIdx.x >= kWarp) {
        return;
    } else if (I.kind == kKindStencil) {
        // the residual of every sweep the launch ran
        for (int ph = lane; ph < I.n_sweeps; ph += kWarp)
            static_cast<float *>(I.o0)[I.sweep0 + round + ph] = __uint_as_float(atomicExch(I.acc + ph, 0u));
    } else {
        // lane l owns bins 8l .. 8l+7: local prefix, then a shuffle scan of
        // the lane totals
        unsigned int c[8], tot = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = atomicExch(I.acc + 8 * lane + k, 0u);
            static_cast<uint32_t *>(I.o0)[8 * lane + k] = c[k];
            tot += c[k];
        }
        unsigned int incl = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (I.o1) {
            unsigned int run = incl - tot;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                static_cast<uint32_t *>(I.o1)[8 * lane + k] = run;
                run += c[k];
            }
        }
    }
}

void describe_instance(const hx_ctx *ctx, const hx_task &t, BInst *out, int64_t *partials, int64_t *acc_words) {
    BInst &I = *out;
    memset(&I, 0, sizeof I);
    I.kind = t.kind;
    *partials = 0;
    *acc_words = 0;
    if (t.kind == HX_TASK_MAP_REDUCE) {
        const auto &m = t.u.mr;
        I.n = m.n;
        I.a = m.a;
        I.plan = mr_plan(m.n > 0 ? m.n : 1, ctx->tune.map_vecs[size_class(m.n)]);
        I.plan.n = m.n;
        I.tiles = m.n > 0 ? I.plan.tiles : 0;
        I.vec = (((uintptr_t)m.x | (uintptr_t)m.y | (uintptr_t)m.out) & 15u) == 0;
        I.in0 = m.x; I.in1 = m.y; I.o0 = m.out; I.o1 = m.sum; I.o2 = m.sum64;
        I.run_len = ctx->tune.batch_map_run;
        *partials = I.tiles;
    } else if (t.kind == HX_TASK_STENCIL2D) {
        const auto &s = t.u.st;
        I.nx = s.nx; I.ny = s.ny; I.iters = s.iters;
        I.n = (int64_t)s.nx * s.ny;
        I.vec = (s.nx % 4 == 0) && ((((uintptr_t)s.u0 | (uintptr_t)s.u1) & 15u) == 0);
        const int width = 128;   // both stencil paths cover 128 columns per warp block
        I.tiles_x = (s.nx + width - 1) / width;
        I.tiles_y = (s.ny + kBatchStRows - 1) / kBatchStRows;
        I.tiles = s.iters > 0 ? (int64_t)I.tiles_x * I.tiles_y : 0;
        I.in0 = s.u0; I.in1 = s.u1; I.o0 = s.resid;
        I.run_len = ctx->tune.batch_stencil_run;
        *acc_words = 1;
    } else {
        const auto &h = t.u.hi;
        I.n = h.n;
        I.tiles = h.n > 0 ? (h.n + kBHiTile - 1) / kBHiTile : 0;
        I.in0 = h.v; I.o0 = h.bins; I.o1 = h.scan;
        I.run_len = 1;
        *acc_words = kHiBins;
    }
    I.n_sweeps = 1;
    I.t_first = 0;
    I.t_count = I.tiles;
}

hx_status launch_batch_round(const hx_ctx *ctx, const BInst *d_insts, uint32_t n_inst, const uint32_t *d_cta_prefix,
                             const uint32_t *d_run_prefix, const uint32_t *d_pairs, uint32_t n_pairs, uint32_t n_cta,
                             uint32_t n_runs, int round, unsigned int *d_ctrl, BatchSync sync, cudaStream_t stream) {
    if (n_cta == 0 && n_runs == 0) return HX_OK;
    if (take_injected_failure(ctx)) return fail(HX_ERR_CUDA, "batched launch: injected launch failure (test hook)");
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    // never more CTAs than the device holds at once: the multi-sweep waits
    // rely on every CTA of the launch being resident
    const int multi = d_pairs ? 1 : 0;
    const int64_t cap = (int64_t)ctx->num_sms * ctx->batch_ctas_per_sm[multi][n_cta > 0 ? 1 : 0];
    const int64_t want = std::max<int64_t>(n_cta, ((int64_t)n_runs + kBatchThreads / kWarp - 1) / (kBatchThreads / kWarp));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(cap, want));
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = n_cta > 0 ? kHiSmemBytes : 0;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = multi ? cudaLaunchKernelEx(&cfg, batch_kernel<true>, d_insts, n_inst, d_cta_prefix, d_run_prefix,
                                               d_pairs, n_pairs, round, d_ctrl, sync)
                          : cudaLaunchKernelEx(&cfg, batch_kernel<false>, d_insts, n_inst, d_cta_prefix, d_run_prefix,
                                               d_pairs, n_inst, round, d_ctrl, sync);
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
    cfg.gridDim = dim3(n_inst);
    cfg.dynamicSmemBytes = 0;
    e = cudaLaunchKernelEx(&cfg, batch_final_kernel, d_insts, n_inst, d_cta_prefix, multi ? nullptr : d_run_prefix,
                           round, d_ctrl);
    if (e != cudaSuccess) return cuda_fail(e, "batched final launch");
    return HX_OK;
}

size_t task_footprint(const hx_task &t) {
    if (t.kind == HX_TASK_MAP_REDUCE) {
        const size_t n = (size_t)(t.u.mr.n > 0 ? t.u.mr.n : 0);
        return n * 4 * (t.u.mr.out ? 3 : 2) + 16;
    }
    if (t.kind == HX_TASK_STENCIL2D)
        return (size_t)t.u.st.nx * t.u.st.ny * 8 + (size_t)(t.u.st.iters > 0 ? t.u.st.iters : 0) * 4;
    return (size_t)(t.u.hi.n > 0 ? t.u.hi.n : 0) + 2048;
}

hx_status batch_setup(hx_ctx *ctx) {
    const void *fns[2] = {(const void *)batch_kernel<false>, (const void *)batch_kernel<true>};
    cudaError_t e = cudaSuccess;
    for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
        e = cudaFuncSetAttribute(fns[m], cudaFuncAttributeMaxDynamicSharedMemorySize, kHiSmemBytes);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[m], kBatchThreads, i ? kHiSmemBytes : 0);
            ctx->batch_ctas_per_sm[m][i] = occ > 0 ? occ : 1;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "hx_create: batch kernel set-up");
    return HX_OK;
}

HX_CHECKS_READER(checks_batch)

}  // namespace hx

struct hx_batch {
    hx_ctx *ctx = nullptr;
    int rounds = 0;
    bool multi = false;                    // one launch runs every sweep of every stencil instance
    uint32_t n_inst = 0;
    uint32_t n_pairs = 0;                  // multi: (instance, sweep) pairs of the launch
    std::vector<uint32_t> n_cta, n_runs;   // per round: CTA chunks, warp runs
    std::vector<hx::BInst> insts;          // host copy of the descriptors (hx_batch_describe)
    void *d_mem = nullptr;
    hx::BInst *d_insts = nullptr;
    uint32_t *d_prefix = nullptr;          // per round: CTA prefix (n_inst + 1), run prefix (n_inst + 1);
                                           // multi: CTA prefix (n_inst + 1), run prefix (n_pairs + 1)
    uint32_t *d_pairs = nullptr;           // multi: the pair list
    unsigned int *d_ctrl = nullptr;        // run counter (reset by each launch)
    unsigned int *err_h = nullptr;         // host-mapped error word of the bounded waits
    unsigned int *err_d = nullptr;
    long long wait_ns = hx::kDefaultWaitNs;
};

namespace hx {

hx_status validate_task(const hx_task &t, int idx, const char *who) {
    char where[96];
    snprintf(where, sizeof where, "%s: task %d: ", who, idx);
    switch (t.kind) {
    case HX_TASK_MAP_REDUCE: {
        const auto &m = t.u.mr;
        if (m.n < 0 || m.n > HX_MAP_REDUCE_MAX_N) return fail(HX_ERR_INVALID, std::string(where) + "n out of range");
        if (!m.sum) return fail(HX_ERR_INVALID, std::string(where) + "sum is NULL");
        if (m.n > 0 && (!m.x || !m.y)) return fail(HX_ERR_INVALID, std::string(where) + "x or y is NULL");
        if ((((uintptr_t)m.x | (uintptr_t)m.y | (uintptr_t)m.out) & 3u) != 0)
            return fail(HX_ERR_INVALID, std::string(where) + "fp32 buffers must be 4-byte aligned");
        return HX_OK;
    }
    case HX_TASK_STENCIL2D: {
        const auto &s = t.u.st;
        if (s.nx < 1 || s.ny < 1 || s.nx > 65536 || s.ny > 65536 || (int64_t)s.nx * s.ny > ((int64_t)1 << 31))
            return fail(HX_ERR_INVALID, std::string(where) + "grid size out of range");
        if (s.iters < 0 || s.iters > kMaxSweeps) return fail(HX_ERR_INVALID, std::string(where) + "iters out of range");
        if (!s.u0 || !s.u1) return fail(HX_ERR_INVALID, std::string(where) + "grid pointer is NULL");
        if (s.iters > 0 && !s.resid) return fail(HX_ERR_INVALID, std::string(where) + "resid is NULL");
        if ((((uintptr_t)s.u0 | (uintptr_t)s.u1) & 3u) != 0)
            return fail(HX_ERR_INVALID, std::string(where) + "grids must be 4-byte aligned");
        const size_t bytes = (size_t)s.nx * s.ny * sizeof(float);
        if ((uintptr_t)s.u0 < (uintptr_t)s.u1 + bytes && (uintptr_t)s.u1 < (uintptr_t)s.u0 + bytes)
            return fail(HX_ERR_INVALID, std::string(where) + "u0 and u1 overlap");
        return HX_OK;
    }
    case HX_TASK_HISTOGRAM: {
        const auto &h = t.u.hi;
        if (h.n < 0 || h.n > HX_HISTOGRAM_MAX_N) return fail(HX_ERR_INVALID, std::string(where) + "n out of range");
        if (!h.bins) return fail(HX_ERR_INVALID, std::string(where) + "bins is NULL");
        if (h.n > 0 && !h.v) return fail(HX_ERR_INVALID, std::string(where) + "v is NULL");
        if ((((uintptr_t)h.bins | (uintptr_t)h.scan) & 3u) != 0)
            return fail(HX_ERR_INVALID, std::string(where) + "bins must be 4-byte aligned");
        return HX_OK;
    }
    default:
        return fail(HX_ERR_INVALID, std::string(where) + "unknown task kind");
    }
}

}  // namespace hx

namespace {

// Releases a partly built plan.
void free_plan(hx_batch *b) {
    if (!b) return;
    if (b->d_mem) cudaFree(b->d_mem);
    if (b->err_h) cudaFreeHost(b->err_h);
    delete b;
}

}  // namespace

extern "C" hx_status hx_batch_plan_ex(hx_ctx *ctx, const hx_task *tasks, int32_t n_tasks, int32_t flags,
                                      hx_batch **out, int32_t *out_rounds) {
    using namespace hx;
    if (!ctx || !out) return fail(HX_ERR_INVALID, "hx_batch_plan: ctx or out is NULL");
    *out = nullptr;
    if (n_tasks < 0 || (n_tasks > 0 && !tasks)) return fail(HX_ERR_INVALID, "hx_batch_plan: bad task list");
    if ((flags & ~(HX_BATCH_ROUNDS | HX_BATCH_ONE_LAUNCH)) || flags == (HX_BATCH_ROUNDS | HX_BATCH_ONE_LAUNCH))
        return fail(HX_ERR_INVALID, "hx_batch_plan: unknown or conflicting flags");
    if ((uint32_t)n_tasks >= kMaxPairInstances) return fail(HX_ERR_INVALID, "hx_batch_plan: too many tasks");
    for (int i = 0; i < n_tasks; ++i) {
        hx_status st = validate_task(tasks[i], i, "hx_batch_plan");
        if (st != HX_OK) return st;
    }
    std::vector<BInst> insts(n_tasks);
    int max_iters = 0;
    int64_t multi_sweep_bytes = 0;
    for (int i = 0; i < n_tasks; ++i) {
        int64_t np = 0, na = 0;
        describe_instance(ctx, tasks[i], &insts[i], &np, &na);
        if (insts[i].tiles > 0xffffffffll) return fail(HX_ERR_INVALID, "hx_batch_plan: instance too large");
        if (insts[i].kind == kKindStencil) max_iters = std::max(max_iters, insts[i].iters);
        if (insts[i].kind == kKindStencil && insts[i].iters > 1 && insts[i].tiles > 0)
            multi_sweep_bytes += 8 * (int64_t)insts[i].nx * insts[i].ny;
    }
    // Several sweeps per stencil instance run in one launch unless the caller
    // asks for rounds (round r = sweep r of every instance, one launch each),
    // or, by default, when the multi-sweep instances move more than
    // kOneLaunchMaxSweepBytes per sweep.  (An instance's sweep offset is
    // stored in 8 bits of its pair entries: batches with more than 255 sweeps
    // run as rounds.)
    const bool multi = max_iters > 1 && max_iters <= 255 && !(flags & HX_BATCH_ROUNDS) &&
                       ((flags & HX_BATCH_ONE_LAUNCH) || multi_sweep_bytes <= kOneLaunchMaxSweepBytes);
    int rounds = n_tasks > 0 ? 1 : 0;
    if (!multi) rounds = std::max(rounds, max_iters);
    int64_t n_partials = 0, n_acc = 0;
    for (BInst &I : insts) {
        if (I.kind == kKindMap) n_partials += I.tiles;
        else if (I.kind == kKindHist) n_acc += kHiBins;
        else {
            if (multi && I.iters > 1) I.n_sweeps = I.iters;
            n_acc += I.n_sweeps + (I.n_sweeps > 1 ? I.tiles : 0);   // one max per sweep, one progress word per block
        }
    }
    if (multi) {
        // Run length of the multi-sweep instances: long runs mean fewer waits
        // and publications (up to kMultiSweepRun blocks), but an instance's
        // next sweep waits for this one, so a sweep of the batch needs about
        // two runs per resident warp to keep the device busy.
        int64_t blocks = 0;
        for (const BInst &I : insts)
            if (I.n_sweeps > 1) blocks += I.tiles;
        const int64_t warps = (int64_t)ctx->num_sms * ctx->batch_ctas_per_sm[1][0] * (kBatchThreads / kWarp);
        const int run = (int)std::max<int64_t>(1, std::min<int64_t>(kMultiSweepRun, blocks / (2 * warps)));
        for (BInst &I : insts)
            if (I.n_sweeps > 1) I.run_len = run;
    }
    // Prefix sums of each launch's work.  Rounds: per round r, the CTA
    // prefix and the run prefix over instances (round 0 holds the one-pass
    // instances; stencil sweep r of each instance goes to round r).  Multi:
    // one launch; CTA prefix over instances, run prefix over the pair list:
    // every instance's first pass, then each later sweep, instances in the
    // same order within every sweep, so a block and the blocks it waits for
    // are about a whole sweep of work apart.
    const size_t stride = (size_t)n_tasks + 1;
    std::vector<uint32_t> prefix, pairs;
    std::vector<uint32_t> round_cta(rounds), round_runs(rounds);
    if (!multi) {
        prefix.assign((size_t)rounds * 2 * stride, 0u);
        for (int r = 0; r < rounds; ++r) {
            uint32_t *cp = prefix.data() + (size_t)r * 2 * stride, *rp = cp + stride;
            uint64_t c = 0, w = 0;
            for (int i = 0; i < n_tasks; ++i) {
                cp[i] = (uint32_t)c;
                rp[i] = (uint32_t)w;
                const BInst &I = insts[i];
                const bool active = (I.kind == kKindStencil) ? (r < I.iters) : (r == 0);
                if (active) {
                    c += inst_ctas(I);
                    w += inst_runs(I);
                }
            }
            if (c > 0xffffffffull || w > 0xffffffffull)
                return fail(HX_ERR_INVALID, "hx_batch_plan: too many work items");
            cp[n_tasks] = (uint32_t)c;
            rp[n_tasks] = (uint32_t)w;
            round_cta[r] = (uint32_t)c;
            round_runs[r] = (uint32_t)w;
        }
    } else {
        std::vector<uint32_t> cp(stride, 0u), rp;
        uint64_t c = 0, w = 0;
        for (int i = 0; i < n_tasks; ++i) {
            cp[i] = (uint32_t)c;
            c += inst_ctas(insts[i]);
            pairs.push_back(make_pair((uint32_t)i, 0u));
        }
        cp[n_tasks] = (uint32_t)c;
        for (int ph = 1; ph < max_iters; ++ph)
            for (int i = 0; i < n_tasks; ++i)
                if (ph < insts[i].n_sweeps) pairs.push_back(make_pair((uint32_t)i, (uint32_t)ph));
        for (uint32_t pr : pairs) {
            rp.push_back((uint32_t)w);
            w += inst_runs(insts[pr & (kMaxPairInstances - 1u)]);
        }
        rp.push_back((uint32_t)w);
        if (c > 0xffffffffull || w > 0xffffffffull || pairs.size() > 0xffffffffull)
            return fail(HX_ERR_INVALID, "hx_batch_plan: too many work items");
        prefix = cp;
        prefix.insert(prefix.end(), rp.begin(), rp.end());
        round_cta[0] = (uint32_t)c;
        round_runs[0] = (uint32_t)w;
    }

    // One device allocation: insts | prefixes | pairs | partials | accumulators | run counter.
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t off_pre = align(sizeof(BInst) * insts.size());
    const size_t off_pairs = off_pre + align(sizeof(uint32_t) * prefix.size());
    const size_t off_part = off_pairs + align(sizeof(uint32_t) * pairs.size());
    const size_t off_acc = off_part + align(sizeof(float2) * n_partials);
    const size_t off_ctrl = off_acc + align(sizeof(unsigned int) * n_acc);
    const size_t total = off_ctrl + 256;
    DeviceGuard g(ctx->device);
    hx_batch *b = new (std::nothrow) hx_batch();
    if (!b) return fail(HX_ERR_NOMEM, "hx_batch_plan: host allocation failed");
    b->ctx = ctx;
    b->rounds = rounds;
    b->multi = multi;
    b->n_inst = (uint32_t)n_tasks;
    b->n_pairs = multi ? (uint32_t)pairs.size() : (uint32_t)n_tasks;
    b->n_cta = round_cta;
    b->n_runs = round_runs;
    cudaError_t e = cudaMalloc(&b->d_mem, total);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&b->err_h), 64, cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *b->err_h = 0u;
        e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&b->err_d), b->err_h, 0);
    }
    if (e != cudaSuccess) {
        free_plan(b);
        return cuda_fail(e, "hx_batch_plan: allocation");
    }
    char *base = static_cast<char *>(b->d_mem);
    b->d_insts = reinterpret_cast<BInst *>(base);
    b->d_prefix = reinterpret_cast<uint32_t *>(base + off_pre);
    b->d_pairs = multi ? reinterpret_cast<uint32_t *>(base + off_pairs) : nullptr;
    b->d_ctrl = reinterpret_cast<unsigned int *>(base + off_ctrl);
    int64_t pcur = 0, acur = 0;
    unsigned int *acc_base = reinterpret_cast<unsigned int *>(base + off_acc);
    for (BInst &I : insts) {
        if (I.kind == kKindMap) {
            I.partials = reinterpret_cast<float2 *>(base + off_part) + pcur;
            pcur += I.tiles;
        } else if (I.kind == kKindStencil) {
            I.acc = acc_base + acur;
            I.done = I.n_sweeps > 1 ? I.acc + I.n_sweeps : nullptr;
            acur += I.n_sweeps + (I.n_sweeps > 1 ? I.tiles : 0);
        } else {
            I.acc = acc_base + acur;
            acur += kHiBins;
        }
    }
    e = cudaMemset(b->d_mem, 0, total);
    if (e == cudaSuccess && !insts.empty())
        e = cudaMemcpy(b->d_insts, insts.data(), sizeof(BInst) * insts.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !prefix.empty())
        e = cudaMemcpy(b->d_prefix, prefix.data(), sizeof(uint32_t) * prefix.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !pairs.empty() && multi)
        e = cudaMemcpy(b->d_pairs, pairs.data(), sizeof(uint32_t) * pairs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_plan(b);
        return cuda_fail(e, "hx_batch_plan: upload");
    }
    // Instances with no tiles still owe their outputs (n == 0 sums, empty
    // histograms): write those directly now, they do not depend on inputs.
    for (int i = 0; i < n_tasks; ++i) {
        const hx_task &t = tasks[i];
        if (t.kind == HX_TASK_MAP_REDUCE && t.u.mr.n == 0) {
            const float z = 0.0f;
            const double z64 = 0.0;
            e = cudaMemcpy(t.u.mr.sum, &z, sizeof z, cudaMemcpyHostToDevice);
            if (e == cudaSuccess && t.u.mr.sum64) e = cudaMemcpy(t.u.mr.sum64, &z64, sizeof z64, cudaMemcpyHostToDevice);
        } else if (t.kind == HX_TASK_HISTOGRAM && t.u.hi.n == 0) {
            e = cudaMemset(t.u.hi.bins, 0, 256 * sizeof(uint32_t));
            if (e == cudaSuccess && t.u.hi.scan) e = cudaMemset(t.u.hi.scan, 0, 256 * sizeof(uint32_t));
        }
        if (e != cudaSuccess) {
            free_plan(b);
            return cuda_fail(e, "hx_batch_plan: empty instance outputs");
        }
    }
    b->insts = insts;
    *out = b;
    if (out_rounds) *out_rounds = rounds;
    if (const char *dump = getenv("HX_DUMP_PLAN"); dump && dump[0] == '1') {
        size_t need = 0;
        hx_batch_describe(b, nullptr, 0, &need);
        std::string text(need, '\0');
        hx_batch_describe(b, text.data(), need, nullptr);
        fputs(text.c_str(), stderr);
    }
    return HX_OK;
}

extern "C" hx_status hx_batch_describe(const hx_batch *b, char *buf, size_t len, size_t *needed) {
    using namespace hx;
    if (!b || (len > 0 && !buf)) return fail(HX_ERR_INVALID, "hx_batch_describe: bad arguments");
    std::string t;
    char line[256];
    uint64_t runs = 0, ctas = 0;
    for (int r = 0; r < b->rounds; ++r) {
        runs += b->n_runs[r];
        ctas += b->n_cta[r];
    }
    snprintf(line, sizeof line, "hx batch plan: %u instances, %s, %d launch%s of the batched kernel (each followed by "
             "its final combine), %llu warp runs, %llu CTA items\n", b->n_inst,
             b->multi ? "every sweep in one launch" : (b->rounds > 1 ? "one launch per sweep (rounds)" : "one pass"),
             b->rounds, b->rounds == 1 ? "" : "es", (unsigned long long)runs, (unsigned long long)ctas);
    t += line;
    if (b->multi) {
        snprintf(line, sizeof line, "  work order: %u (instance, sweep) pairs, sweep-major; a block of sweep s waits "
                 "for itself and its 4 neighbours in sweep s-1 (bounded, %.3f s)\n", b->n_pairs, b->wait_ns * 1e-9);
        t += line;
    }
    static const char *kinds[3] = {"map->reduce", "stencil", "histogram"};
    for (uint32_t i = 0; i < b->n_inst; ++i) {
        const BInst &I = b->insts[i];
        if (I.kind == kKindMap)
            snprintf(line, sizeof line, "  [%u] %s n=%lld tiles=%lld x %lld elements, runs of %d, %s path\n", i,
                     kinds[I.kind], (long long)I.n, (long long)I.tiles, (long long)I.plan.tile_elems, I.run_len,
                     I.vec ? "float4" : "element");
        else if (I.kind == kKindStencil)
            snprintf(line, sizeof line, "  [%u] %s %d x %d, %d sweep%s%s, %lld blocks of %d x 128 per sweep, runs of "
                     "%d, %s path\n", i, kinds[I.kind], I.ny, I.nx, I.iters, I.iters == 1 ? "" : "s",
                     I.n_sweeps > 1 ? " in one launch" : (I.iters > 1 ? " as rounds" : ""), (long long)I.tiles,
                     kBatchStRows, I.run_len, I.vec ? "float4" : (b->multi && I.n_sweeps > 1 ? "lane-strided" : "element"));
        else
            snprintf(line, sizeof line, "  [%u] %s n=%lld bytes, %lld CTA chunks of %lld bytes\n", i, kinds[I.kind],
                     (long long)I.n, (long long)I.tiles, (long long)kBHiTile);
        t += line;
    }
    if (needed) *needed = t.size() + 1;
    if (len > 0) {
        const size_t n = std::min(len - 1, t.size());
        memcpy(buf, t.data(), n);
        buf[n] = '\0';
    }
    return HX_OK;
}

extern "C" hx_status hx_batch_plan(hx_ctx *ctx, const hx_task *tasks, int32_t n_tasks, hx_batch **out,
                                   int32_t *out_rounds) {
    return hx_batch_plan_ex(ctx, tasks, n_tasks, 0, out, out_rounds);
}

extern "C" hx_status hx_batch_launch(hx_batch *b, hx_stream_t stream) {
    using namespace hx;
    if (!b) return fail(HX_ERR_INVALID, "hx_batch_launch: batch is NULL");
    DeviceGuard g(b->ctx->device);
    const BatchSync sync{b->err_d, b->wait_ns};
    if (b->multi)
        return launch_batch_round(b->ctx, b->d_insts, b->n_inst, b->d_prefix, b->d_prefix + b->n_inst + 1, b->d_pairs,
                                  b->n_pairs, b->n_cta[0], b->n_runs[0], 0, b->d_ctrl, sync, (cudaStream_t)stream);
    const size_t stride = (size_t)b->n_inst + 1;
    for (int r = 0; r < b->rounds; ++r) {
        const uint32_t *cp = b->d_prefix + (size_t)r * 2 * stride;
        hx_status st = launch_batch_round(b->ctx, b->d_insts, b->n_inst, cp, cp + stride, nullptr, b->n_inst,
                                          b->n_cta[r], b->n_runs[r], r, b->d_ctrl, sync, (cudaStream_t)stream);
        if (st != HX_OK) return st;
    }
    return HX_OK;
}

extern "C" hx_status hx_batch_status(hx_batch *b) {
    using namespace hx;
    if (!b) return fail(HX_ERR_INVALID, "hx_batch_status: batch is NULL");
    const unsigned int e = __atomic_exchange_n(b->err_h, 0u, __ATOMIC_ACQ_REL);
    if (e == (unsigned int)HX_ERR_TIMEOUT)
        return fail(HX_ERR_TIMEOUT, "hx_batch_status: a sweep's wait ran out of time; results are not valid");
    return HX_OK;
}

extern "C" hx_status hx_debug_batch_stall(hx_batch *b, int32_t task, int64_t wait_limit_ns) {
    using namespace hx;
    if (!b || task < 0 || (uint32_t)task >= b->n_inst || wait_limit_ns < 0)
        return fail(HX_ERR_INVALID, "hx_debug_batch_stall: bad arguments");
    DeviceGuard g(b->ctx->device);
    const int one = 1;
    cudaError_t e = cudaMemcpy(reinterpret_cast<char *>(b->d_insts + task) + offsetof(BInst, stall), &one, sizeof one,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "hx_debug_batch_stall");
    b->wait_ns = wait_limit_ns;
    return HX_OK;
}

extern "C" void hx_batch_free(hx_batch *b) {
    if (!b) return;
    hx::DeviceGuard g(b->ctx->device);
    free_plan(b);
}

extern "C" hx_status hx_batch_submit(hx_ctx *ctx, const hx_task *tasks, int32_t n_tasks, hx_stream_t stream,
                                     uint64_t *ticket_out) {
    using namespace hx;
    if (!ctx || !ticket_out) return fail(HX_ERR_INVALID, "hx_batch_submit: ctx or ticket_out is NULL");
    hx_batch *b = nullptr;
    hx_status st = hx_batch_plan(ctx, tasks, n_tasks, &b, nullptr);
    if (st != HX_OK) return st;
    st = hx_batch_launch(b, stream);
    if (st != HX_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        hx_batch_free(b);
        return st;
    }
    DeviceGuard g(ctx->device);
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize((cudaStream_t)stream);
        hx_batch_free(b);
        return cuda_fail(e, "hx_batch_submit: completion event");
    }
    const uint64_t ticket = ctx->next_ticket++;
    ctx->pending[ticket] = {b, ev};
    *ticket_out = ticket;
    return HX_OK;
}

extern "C" hx_status hx_batch_query(hx_ctx *ctx, uint64_t ticket) {
    using namespace hx;
    if (!ctx) return fail(HX_ERR_INVALID, "hx_batch_query: ctx is NULL");
    auto it = ctx->pending.find(ticket);
    if (it == ctx->pending.end()) return fail(HX_ERR_INVALID, "hx_batch_query: unknown ticket");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaEventQuery(it->second.second);
    if (e == cudaErrorNotReady) return HX_ERR_BUSY;
    cudaEventDestroy(it->second.second);
    const hx_status waits = e == cudaSuccess ? hx_batch_status(it->second.first) : HX_OK;
    hx_batch_free(it->second.first);
    ctx->pending.erase(it);
    if (e != cudaSuccess) return cuda_fail(e, "hx_batch_query: device work failed");
    return waits;
}
