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
    unsigned int *done; // stencil with n_sweeps > 1: blocks finished, per sweep but the last
    int stall;          // test hook (hx_debug_batch_stall): this instance's waits are never satisfied
    int pad3;
};

// Bounded waits of a launch that runs several sweeps of an instance: a run
// of sweep s waits until every block of sweep s - 1 of its instance is done.
// A wait gives up after limit_ns nanoseconds of %globaltimer; the kernel
// then records HX_ERR_TIMEOUT in *err (host-mapped memory, read by the host
// once the launch has completed) and carries on, so no wait is unbounded and
// no later wait depends on the one that gave up.
struct BatchSync {
    unsigned int *err;
    long long limit_ns;
};
constexpr long long kDefaultWaitNs = 1000000000ll;   // 1 s
// Blocks per warp run (at most) of a stencil instance that runs several
// sweeps in one launch: every run of such an instance waits for, and
// publishes to, a sweep counter, so longer runs mean fewer round trips, while
// a sweep cannot use more warps than it has runs (the planner shortens runs
// until a sweep of the launch has about two per resident warp).  Measured on
// the 512-instance, 20-sweep batch (B300): 4 blocks 4.51 ms, 8 blocks
// 4.41 ms, 16 blocks 4.55 ms, 32 blocks 4.80 ms.
constexpr int kMultiSweepRun = 8;
// A plan runs several sweeps of its instances in one launch by default only
// if at least this many stencil instances have several sweeps.  Measured on
// B300, 20 sweeps: one 4096^2 grid took 0.76 ms in one launch against
// 0.55 ms as rounds, while 8 grids of sides 1024-4096 took 1.07 ms against
// 1.23 ms.
constexpr int kMinMultiInstances = 4;
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

// Work items of one launch in the order workers take them: every instance's
// sweep-0 work (and all map and histogram work), then the second sweep of
// each instance that runs several, and so on.  Entry k of a launch's pair list
// names (instance, sweep offset) as instance | offset << 24; the run prefix
// then has one entry per pair plus a total.  A launch whose stencils run one
// sweep each has no pair list: entry k is instance k.
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
