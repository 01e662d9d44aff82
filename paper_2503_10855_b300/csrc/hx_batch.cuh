// hx_batch.cuh -- the batched kernel's work description, shared by the batch
// planner (hx_batch.cu) and the serving engine (hx_serve.cu).
#pragma once

#include <vector>

#include "hx_internal.cuh"

namespace hx {

enum : int { kKindMap = 0, kKindStencil = 1, kKindHist = 2 };

constexpr int kBatchThreads = 256;                               // 8 warps
constexpr int64_t kBHiTile = (int64_t)256 * 1024;                // bytes per histogram item
constexpr int kMaxSweeps = 4096;
static_assert(kBatchThreads == kHiBins, "the histogram finish maps one thread to one bin");
static_assert(kBatchThreads == kMrFoldLanes, "the final combine maps one thread to one virtual lane");


struct BInst {
    int kind;
    int vec;            // map: 16-byte aligned operands; stencil: vector path; hist: unused
    int nx, ny;
    float a;
    int iters;          // stencil sweeps
    int sweep0;         // stencil: sweep index of this launch's round 0
    int64_t n;
    int64_t tiles;      // items per round
    int tiles_x;        // stencil warp blocks across
    int tiles_y;        // stencil warp blocks down
    int run_len;        // map / stencil: tiles per warp run
    int n_sweeps;       // stencil: sweeps sweep0 .. sweep0 + n_sweeps - 1 run in this launch (1 otherwise)
    int64_t t_first;    // this launch's slice: tiles (histogram: chunks) [t_first, t_first + t_count)
    int64_t t_count;
    MrPlan plan;
    const void *in0;    // map x | stencil u0 | hist v
    const void *in1;    // map y | stencil u1
    void *o0;           // map out | stencil resid | hist bins
    void *o1;           // map sum | hist scan
    void *o2;           // map sum64
    float2 *partials;   // map tile partials (hi, lo)
    unsigned int *acc;  // stencil: max bits, one word per sweep of the launch; hist: 256 bins
    unsigned int *done; // stencil with n_sweeps > 1: one progress word per block (tiles of them), the
                        // sweeps of this launch the block has finished; zero between launches
    int stall;          // test hook (hx_debug_batch_stall): this instance's waits are never satisfied
    int pad3;
};

// Bounded waits of a launch that runs several sweeps of an instance: a block
// of sweep s waits until it and its four neighbouring blocks (north, south,
// west, east) have finished sweep s - 1 -- they wrote the cells it reads,
// and they read the cells it overwrites (the grids alternate).  A wait gives
// up after limit_ns nanoseconds of %globaltimer; the kernel then records
// HX_ERR_TIMEOUT in *err (host-mapped memory, read by the host once the
// launch has completed) and carries on, so no wait is unbounded and no later
// wait depends on the one that gave up.
struct BatchSync {
    unsigned int *err;
    long long limit_ns;
};
constexpr long long kDefaultWaitNs = 1000000000ll;   // 1 s
// Blocks per warp run (at most) of a stencil instance that runs several
// sweeps in one launch: every run of such an instance waits for, and
// publishes, its blocks' progress, so longer runs mean fewer round trips,
// while a sweep cannot use more warps than it has runs (the planner shortens
// runs until a sweep of the launch has about two per resident warp).
constexpr int kMultiSweepRun = 8;
// A plan runs several sweeps of its instances in one launch by default only
// if its multi-sweep instances move at most this many bytes per sweep.  With
// larger sweeps a launch per sweep hides its launch gaps and its one-sweep
// blocks (read-only loads through L1) are cheaper.  Measured on B300, 20
// sweeps, one launch against rounds: one 4096^2 grid 0.479 against 0.544 ms,
// 8 grids of sides 1024-4096 1.09 against 1.22 ms, 64 grids of 32-2048 1.07
// against 1.19 ms, and 252 grids of 32-2048 (1 GB per sweep) 4.27 against
// 3.98 ms.
constexpr int64_t kOneLaunchMaxSweepBytes = (int64_t)512 << 20;
constexpr int kMaxStepSweeps = 128;                 // sweeps of one request in one serving step


// Checks one task against the rules of its standalone call.
hx_status validate_task(const hx_task &t, int idx, const char *who);

// Describes one task as an instance (no workspace pointers yet) and reports
// the workspace it needs: tile partials and accumulator words.
void describe_instance(const hx_ctx *ctx, const hx_task &t, BInst *out, int64_t *partials, int64_t *acc_words);

// Work items of one launch of instance I (its slice [t_first, t_first +
// t_count)): warp runs for map->reduce and stencil, CTA chunks for histogram.
inline uint32_t inst_runs(const BInst &I) {
    return I.kind == kKindHist ? 0u : (uint32_t)((I.t_count + I.run_len - 1) / I.run_len);
}
inline uint32_t inst_ctas(const BInst &I) { return I.kind == kKindHist ? (uint32_t)I.t_count : 0u; }

// Work items of one launch in the order workers take them, listed as
// (instance, sweep offset) pairs: a pair's work waits only for pairs listed
// before it (an instance's sweep s - 1 comes before its sweep s).  Entry k of
// a launch's pair list names (instance, sweep offset) as instance | offset
// << 24; the run prefix then has one entry per pair plus a total.  A launch
// whose stencils run one sweep each has no pair list: entry k is instance k.
inline uint32_t make_pair(uint32_t inst, uint32_t phase) { return inst | (phase << 24); }
constexpr uint32_t kMaxPairInstances = 1u << 24;

// Launches the batched kernel (n_inst instances; exclusive prefix sums of
// their CTA chunks, n_inst + 1 entries, and of their warp runs per pair,
// n_pairs + 1 entries, on the device; totals n_cta and n_runs; d_pairs NULL
// when every stencil instance runs one sweep, and then n_pairs == n_inst) and
// after it the final-combine kernel for the instances it completes.  d_ctrl:
// a zeroed word the kernels use as the run counter and leave zeroed
// (launches sharing d_ctrl must be ordered, e.g. on one stream).
hx_status launch_batch_round(const hx_ctx *ctx, const BInst *d_insts, uint32_t n_inst, const uint32_t *d_cta_prefix,
                             const uint32_t *d_run_prefix, const uint32_t *d_pairs, uint32_t n_pairs, uint32_t n_cta,
                             uint32_t n_runs, int round, unsigned int *d_ctrl, BatchSync sync, cudaStream_t stream);

// Device bytes a task's buffers occupy (inputs and outputs), for admission.
size_t task_footprint(const hx_task &t);

}  // namespace hx
