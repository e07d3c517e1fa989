// Device side of the batched persistent launch (snlm_batch.cu): the job and
// control records, the bounded dependency waits and the per-K class kernel. Each
// class kernel is instantiated in a translation unit of its own (snlm_batch_k*.cu)
// so that the library's build compiles them in parallel.
#pragma once

#include "snlm_host.h"
#include "snlm_pass_impl.cuh"
#include "snlm_sure_impl.cuh"

namespace snlm {
namespace batch {


constexpr int kKindPass = 0, kKindSolve = 1, kKindCombine = 2;
constexpr int kCombineChunk = 4096;      // pixels per combination unit
constexpr int kMaxClasses = 8;           // K = 1..7 (index K)

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
    int head[kMaxClasses];  // next unit of each class
    int err;                // a bounded wait gave up
    int err_job;
    int pad[6];
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

// Each pass variant is its own (not inlined) function, so that its registers are
// allocated for it alone rather than for the union of six inlined bodies.
template <int K, int DM, bool SURE>
__device__ __noinline__ void pass_unit_variant(const PassArgs &a, int unit, float *smem)
{
    process_tile<K, DM, SURE>(a, unit, smem);
}

template <int K>
__device__ __forceinline__ void run_pass_unit(const BatchJob &j, int unit, float *smem)
{
    const int sel = j.dm * 2 + j.sure;
    switch (sel) {
    case DIST_SLIDE * 2 + 0: pass_unit_variant<K, DIST_SLIDE, false>(j.a, unit, smem); break;
    case DIST_SLIDE * 2 + 1: pass_unit_variant<K, DIST_SLIDE, true>(j.a, unit, smem); break;
    case DIST_BLOCK * 2 + 0: pass_unit_variant<K, DIST_BLOCK, false>(j.a, unit, smem); break;
    case DIST_BLOCK * 2 + 1: pass_unit_variant<K, DIST_BLOCK, true>(j.a, unit, smem); break;
    case DIST_FIR * 2 + 0: pass_unit_variant<K, DIST_FIR, false>(j.a, unit, smem); break;
    default: pass_unit_variant<K, DIST_FIR, true>(j.a, unit, smem); break;
    }
}

// One persistent CTA loop over the units of one K class. unit_job[u] is the job of
// the class's unit u (a table built with the plan). Thread 0 claims the CTA's next
// unit while the CTA works on the current one, so the claim's round trip to L2 is
// hidden; units are still taken in increasing order per CTA, and every unit's
// dependencies lie in earlier jobs, so the lowest unfinished unit is always one
// that some CTA is working on. The job record is copied to shared memory only when
// the job changes (consecutive units usually share it).
template <int K>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 4)
batch_kernel(const BatchJob *__restrict__ jobs, const int *__restrict__ unit_job, int n_units, int cls,
             BatchCtl *ctl, int *done, unsigned long long limit_ns)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(16) BatchJob sj;
    __shared__ int s_unit, s_job, s_fail;
    int next = 0, have = -1;                   // thread 0: claimed next unit; job held in sj
    if (threadIdx.x == 0)
        next = ld_acquire(&ctl->err) == 0 ? atomicAdd(&ctl->head[cls], 1) : n_units;
    for (;;) {
        if (threadIdx.x == 0) {
            int u = next, jb = -1, fail = 0;
            if (u < n_units && ld_acquire(&ctl->err) != 0)
                u = n_units;
            if (u < n_units) {
                jb = unit_job[u];
                const BatchJob &J = jobs[jb];
                if ((J.dep0 >= 0 && !wait_count(done + J.dep0, J.need0, limit_ns)) ||
                    (J.dep1 >= 0 && !wait_count(done + J.dep1, J.need1, limit_ns)))
                    fail = 1;
            }
            if (fail) {
                atomicExch(&ctl->err_job, jb);
                atomicExch(&ctl->err, 1);
                __threadfence();
            }
            s_unit = u;
            s_job = jb;
            s_fail = fail;
        }
        __syncthreads();
        const int u = s_unit;
        if (u >= n_units || s_fail)
            return;
        if (threadIdx.x == 0)
            next = atomicAdd(&ctl->head[cls], 1);
        if (s_job != have) {
            have = s_job;
            const int *src = reinterpret_cast<const int *>(jobs + have);
            int *dst = reinterpret_cast<int *>(&sj);
            for (int i = threadIdx.x; i < (int)(sizeof(BatchJob) / sizeof(int)); i += blockDim.x)
                dst[i] = src[i];
            __syncthreads();
        }
        const int unit = u - sj.unit0;
        if (sj.kind == kKindPass) {
            run_pass_unit<K>(sj, unit, smem);
        } else if (sj.kind == kKindSolve) {
            double rc[kPartials], cr[kPartials];
            double *sh = reinterpret_cast<double *>(smem);
            reduce_records(sj.part_rc, sj.n_rc, sh, rc);
            reduce_records(sj.part_cr, sj.n_cr, sh, cr);
            if (threadIdx.x == 0)
                sure_finish(rc, cr, sj.sigma2, sj.info);
        } else {
            const long long lo = (long long)unit * kCombineChunk;
            combine_range(sj.frc, sj.out, sj.info, lo, min(sj.n_px, lo + kCombineChunk));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + s_job, 1);
        }
    }
}

using BatchFn = void (*)(const BatchJob *, const int *, int, int, BatchCtl *, int *, unsigned long long);

// The class kernel of patch half-width K (defined in snlm_batch_k<K>.cu).
template <int K>
BatchFn batch_kernel_ptr();

}  // namespace batch
}  // namespace snlm

#define SNLM_INSTANTIATE_BATCH_K(KK) \
    template <> snlm::batch::BatchFn snlm::batch::batch_kernel_ptr<KK>() { return snlm::batch::batch_kernel<KK>; }
