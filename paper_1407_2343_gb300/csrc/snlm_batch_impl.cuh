// Device side of the batched persistent launch (snlm_batch.cu): the job and
// control records, the bounded dependency waits and the class kernels: one per
// (K, pass variant) with the pass inlined as in the single-image kernel, and one for
// the solve and combination jobs. The pass class kernels of each K are instantiated
// in a translation unit of their own (snlm_batch_k*.cu) so that the library's build
// compiles them in parallel.
#pragma once

#include "snlm_host.h"
#include "snlm_pass_impl.cuh"
#include "snlm_sure_impl.cuh"

namespace snlm {
namespace batch {


constexpr int kKindPass = 0, kKindSolve = 1, kKindCombine = 2;
constexpr int kCombineChunk = 4096;      // pixels per combination unit
constexpr int kVariants = 6;            // pass variants: distance mode x SURE
constexpr int kVariantMisc = kVariants; // the class of the solve and combination jobs

struct BatchJob {
    PassArgs a;            // pass jobs
    int kind;              // kKind*
    int dm, sure;          // pass variant
    int n_units, unit0;    // class-local queue range
    int dep0, dep1;        // global job indices (-1: none)
    int need0, need1;      // completion counts required from them
    // solve
    const double *part_rc, *part_cr;
    int n_rc, n_cr;
    double sigma2;
    double *info;
    // combination
    const float *frc;
    float *out;
    long long n_px;
};

struct BatchCtl {
    int err;                // a bounded wait gave up
    int err_job;
    int pad[6];
};

// What a CTA needs to start its unit, in one 32-byte record per unit (built with the
// plan): the job, the unit's index inside the job, and the job's dependencies with
// the completion counts they must reach.
struct __align__(16) UnitRec {
    int job, unit;
    int dep0, need0, dep1, need1;
    int pad0, pad1;
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits (bounded) until *ctr >= need; false if the bound was hit.
static __device__ bool wait_count(const int *ctr, int need, unsigned long long limit_ns)
{
    if (need <= 0 || ld_acquire(ctr) >= need)
        return true;
    const unsigned long long t0 = global_ns();
    while (ld_acquire(ctr) < need) {
        if (global_ns() - t0 > limit_ns)
            return false;
        __nanosleep(500);
    }
    return true;
}

// One unit of a class kernel: the grid has one CTA per unit of the class, CTA b
// runs unit b. A class holds jobs of one dependency level, so every job a unit
// depends on belongs to an earlier class, which the stream ran to the end before
// this launch: the dependencies are complete when the CTA starts. The CTA still
// checks the per-job completion counters (a bounded wait, which only an injected
// fault can make run out), and releases its own unit by a counter increment that
// later launches read. work(job, unit, smem) runs the unit; `job` points to the job
// table in global memory, read-only for the launch, so the pass code reads its
// arguments through the read-only path. (A persistent loop over the units held the
// tile's loop-invariant values in registers across units and spilled 0.5-1 KB per
// thread; taking units with an atomic claim put an L2 round trip before every
// unit's work.)
template <typename Work>
__device__ __forceinline__ void run_unit(const BatchJob *__restrict__ jobs, const UnitRec *__restrict__ recs,
                                         BatchCtl *ctl, int *done, unsigned long long limit_ns, float *smem,
                                         Work work)
{
    __shared__ int s_job, s_unit, s_fail;
    if (threadIdx.x == 0) {
        const UnitRec r = recs[blockIdx.x];
        int fail = ld_acquire(&ctl->err) != 0 ? 2 : 0;
        if (fail == 0 && ((r.dep0 >= 0 && !wait_count(done + r.dep0, r.need0, limit_ns)) ||
                          (r.dep1 >= 0 && !wait_count(done + r.dep1, r.need1, limit_ns)))) {
            fail = 1;
            atomicExch(&ctl->err_job, r.job);
            atomicExch(&ctl->err, 1);
            __threadfence();
        }
        s_job = r.job;
        s_unit = r.unit;
        s_fail = fail;
    }
    __syncthreads();
    if (s_fail)
        return;
    const int jb = s_job;
    work(jobs[jb], s_unit, smem);
    __syncthreads();
    if (threadIdx.x == 0)
        atomicAdd(done + jb, 1);
}

// The class kernel of the pass variant (K, DM, SURE): the single-image kernel's tile
// code inlined, with its occupancy.
template <int K, int DM, bool SURE>
__global__ void __launch_bounds__(kWarpsPerCta * 32, pass_min_ctas<K, DM, SURE>())
batch_pass_kernel(const BatchJob *__restrict__ jobs, const UnitRec *__restrict__ recs, BatchCtl *ctl, int *done,
                  unsigned long long limit_ns)
{
    extern __shared__ __align__(16) float smem[];
    run_unit(jobs, recs, ctl, done, limit_ns, smem,
             [](const BatchJob &j, int unit, float *sm) { process_tile<K, DM, SURE>(j.a, unit, sm); });
}

// The class kernel of the solve and combination jobs of SURE.
__global__ void __launch_bounds__(kWarpsPerCta * 32)
batch_misc_kernel(const BatchJob *__restrict__ jobs, const UnitRec *__restrict__ recs, BatchCtl *ctl, int *done,
                  unsigned long long limit_ns);

using BatchFn = void (*)(const BatchJob *, const UnitRec *, BatchCtl *, int *, unsigned long long);

// The pass class kernel of (K, variant), variant = distance mode * 2 + SURE
// (defined in snlm_batch_k<K>.cu).
template <int K>
BatchFn batch_pass_kernel_ptr(int variant);

}  // namespace batch
}  // namespace snlm

#define SNLM_INSTANTIATE_BATCH_K(KK)                                                                  \
    template <>                                                                                       \
    snlm::batch::BatchFn snlm::batch::batch_pass_kernel_ptr<KK>(int variant)                          \
    {                                                                                                 \
        using namespace snlm;                                                                         \
        switch (variant) {                                                                            \
        case DIST_SLIDE * 2 + 0: return batch_pass_kernel<KK, DIST_SLIDE, false>;                     \
        case DIST_SLIDE * 2 + 1: return batch_pass_kernel<KK, DIST_SLIDE, true>;                      \
        case DIST_BLOCK * 2 + 0: return batch_pass_kernel<KK, DIST_BLOCK, false>;                     \
        case DIST_BLOCK * 2 + 1: return batch_pass_kernel<KK, DIST_BLOCK, true>;                      \
        case DIST_FIR * 2 + 0: return batch_pass_kernel<KK, DIST_FIR, false>;                         \
        case DIST_FIR * 2 + 1: return batch_pass_kernel<KK, DIST_FIR, true>;                          \
        default: return nullptr;                                                                      \
        }                                                                                             \
    }
