// Batched separable NLM: many independent images in a few launches over a work
// queue of CTA-sized units (declared in include/snlm.h, snlm_batch_*).
//
// Each image becomes jobs: one per 1-D pass of its order (Alg. 4: rows then
// columns, columns then rows), and for SURE a solve job and combination jobs
// (Eqs. (14), (19), (25)). A job is split into units (kWarpsPerCta lines x one
// tile, exactly the units of the single-image kernels). Jobs are grouped into
// classes by dependency level (a job depends only on jobs of lower levels), then by
// kernel (a pass variant and K, or the solve and combination jobs); each class is
// one launch with one CTA per unit, and the classes run one after another on the
// stream in level order, so every dependency of a unit is complete when its CTA
// starts. The CTAs still check their dependencies' completion counters with a
// bounded wait (a time limit read from %globaltimer), which only an injected fault
// runs out; a CTA that gives up records it in the control block, and the CTAs after
// it do no work.
#include <algorithm>
#include <cstddef>
#include <memory>
#include <numeric>

#include "snlm_host.h"
#include "snlm_batch_impl.cuh"

namespace snlm {
namespace batch {

__global__ void __launch_bounds__(kWarpsPerCta * 32)
batch_misc_kernel(const BatchJob *__restrict__ jobs, const UnitRec *__restrict__ recs, BatchCtl *ctl, int *done,
                  unsigned long long limit_ns)
{
    extern __shared__ __align__(16) float smem[];
    run_unit(jobs, recs, ctl, done, limit_ns, smem, [](const BatchJob &j, int unit, float *sm) {
        if (j.kind == kKindSolve) {
            double rc[kPartials], cr[kPartials];
            double *sh = reinterpret_cast<double *>(sm);
            reduce_records(j.part_rc, j.n_rc, sh, rc);
            reduce_records(j.part_cr, j.n_cr, sh, cr);
            if (threadIdx.x == 0)
                sure_finish(rc, cr, j.sigma2, j.info);
        } else {
            const long long lo = (long long)unit * kCombineChunk;
            combine_range(j.frc, j.out, j.info, lo, min(j.n_px, lo + kCombineChunk));
        }
    });
}

}  // namespace batch

namespace {

using namespace snlm::batch;

// The class kernel of (K, variant): variant = distance mode * 2 + SURE for the
// passes, kVariantMisc for the solve and combination jobs.
BatchFn batch_fn(int K, int variant)
{
    if (variant == kVariantMisc)
        return batch_misc_kernel;
    switch (K) {
    case 1: return batch_pass_kernel_ptr<1>(variant);
    case 2: return batch_pass_kernel_ptr<2>(variant);
    case 3: return batch_pass_kernel_ptr<3>(variant);
    case 4: return batch_pass_kernel_ptr<4>(variant);
    case 5: return batch_pass_kernel_ptr<5>(variant);
    case 6: return batch_pass_kernel_ptr<6>(variant);
    case 7: return batch_pass_kernel_ptr<7>(variant);
    default: return nullptr;
    }
}

// Shared-memory limit and occupancy of a class kernel, cached per (device, kernel,
// bytes): the shared-memory attribute only ever grows, and a serving loop builds a
// plan per step.
cudaError_t class_occupancy(BatchFn fn, int dev, size_t smem, int *occ)
{
    struct Entry {
        int dev;
        BatchFn fn;
        size_t smem;
        int occ;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    static std::vector<Entry> attr;     // (dev, fn) -> the attribute set so far (in .smem)
    std::lock_guard<std::mutex> g(mu);
    for (const Entry &c : cache)
        if (c.dev == dev && c.fn == fn && c.smem == smem) {
            *occ = c.occ;
            return cudaSuccess;
        }
    Entry *slot = nullptr;
    for (Entry &a : attr)
        if (a.dev == dev && a.fn == fn)
            slot = &a;
    if (!slot) {
        attr.push_back(Entry{dev, fn, 0, 0});
        slot = &attr.back();
    }
    if (slot->smem < smem) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        slot->smem = smem;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, kWarpsPerCta * 32, smem);
    if (e == cudaSuccess)
        cache.push_back(Entry{dev, fn, smem, *occ});
    return e;
}

struct ClassInfo {
    int K = 0;                // 0 for the class of the solve and combination jobs
    int variant = 0;
    int j0 = 0, nj = 0;       // job range (global indices, contiguous)
    int n_units = 0;
    int u_off = 0;            // the class's first entry in the unit records
    size_t smem = 0;          // dynamic shared memory the class kernel needs
    size_t smem_launch = 0;   // and launches with (more when CTAs per SM are capped)
    int grid = 0;             // one CTA per unit
};

}  // namespace

int preload_batch()
{
    int n = preload_kernel((const void *)batch_fn(0, kVariantMisc));
    for (int K = 1; K <= 7; ++K)
        for (int v = 0; v < kVariants; ++v)
            n += preload_kernel((const void *)batch_fn(K, v));
    return n;
}

}  // namespace snlm

using namespace snlm;

// A scratch pointer of a job, filled in at upload: field `field` of job `job`
// points `offset` bytes into the scratch area of the workspace.
struct Reloc {
    int job, field;
    size_t offset;
};
enum RelocField { R_SRC, R_DST, R_BLEND, R_DIN, R_DOUT, R_PARTIALS, R_AUXRC, R_PART_RC, R_PART_CR, R_INFO, R_FRC };

struct snlm_batch_plan {
    std::vector<BatchJob> jobs;
    std::vector<ClassInfo> classes;
    std::vector<Reloc> relocs;
    std::vector<UnitRec> unit_recs;   // every unit's record, class after class
    size_t ws_bytes = 0, jobs_off = 0, done_off = 0, ctl_off = 0, scratch_off = 0, units_off = 0;
    snlm_batch_config cfg{};
    void *ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int units = 0;
};

namespace {

size_t max_layout_bytes(int S, int K, bool sure)
{
    return (size_t)warp_layout(S, K, sure, false).per_warp * kWarpsPerCta * sizeof(float);
}

int validate_request(const snlm_request &r)
{
    int rc = check_common(r.H, r.W, r.S, r.K, r.h, r.profile, r.order, r.sigma);
    if (rc != SNLM_OK)
        return rc;
    if (r.K < 1)
        return SNLM_ERR_UNSUPPORTED;
    if (!valid_dtype(r.dtype) || r.pitch < r.W || (long long)r.H * r.pitch >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (!r.img || !r.out)
        return SNLM_ERR_ARG;
    return SNLM_OK;
}

PassArgs pass_args(int axis, int H, int W, const Lines &src, float *dst, int S, int K, double h,
                   int profile, double beta)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.n_lines = axis == 0 ? H : W;
    a.N = axis == 0 ? W : H;
    a.S = S;
    a.c2 = exp2_scale(h);
    a.h2 = (float)(h * h);
    fill_profile(a.g, K, profile, beta);
    a.dst = dst;
    a.out_line_step = axis == 0 ? W : 1;
    a.out_elem_step = axis == 0 ? 1 : W;
    a.aux_f = Lines{nullptr, DT_F32, 0, 0};
    a.aux_rc = Lines{nullptr, DT_F32, 0, 0};
    finish_pass_args(a);
    return a;
}

}  // namespace

extern "C" {

int snlm_batch_plan_create(const snlm_request *reqs, int n, const snlm_batch_config *cfg,
                           snlm_batch_plan **plan_out)
{
    if (!plan_out || n < 1 || !reqs)
        return SNLM_ERR_ARG;
    *plan_out = nullptr;
    for (int i = 0; i < n; ++i) {
        int rc = validate_request(reqs[i]);
        if (rc != SNLM_OK)
            return rc;
    }
    std::unique_ptr<snlm_batch_plan> P(new snlm_batch_plan());
    if (cfg)
        P->cfg = *cfg;
    else
        P->cfg = snlm_batch_config{0, 0, 0, -1};

    // request order inside each level (the queue policy)
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if (P->cfg.queue_order == 1 || P->cfg.queue_order == 2) {
        const bool big_first = P->cfg.queue_order == 1;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const long long pa = (long long)reqs[a].H * reqs[a].W, pb = (long long)reqs[b].H * reqs[b].W;
            return big_first ? pa > pb : pa < pb;
        });
    }

    // Per-request scratch (offsets inside the scratch area): f_r, f_c, f_rc, delta_1,
    // delta_2, partial sums of the two last passes, info.
    struct Proto {
        BatchJob j;
        int level, req;
    };
    std::vector<Proto> protos;
    std::vector<Reloc> relocs;   // job indices refer to `protos` until the final sort
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes, 256);
        return o;
    };
    for (int i = 0; i < n; ++i) {
        const snlm_request &r = reqs[i];
        const double bt = beta_or_default(r.beta, r.K);
        const int dm_img = dist_mode_for(r.dtype, r.profile);
        const int dm_f32 = dist_mode_for(SNLM_F32, r.profile);
        const bool sure = r.order == SNLM_SURE;
        const size_t img = (size_t)r.H * r.W * sizeof(float);
        const size_t o_fr = r.order != SNLM_CR ? take(img) : 0;
        const size_t o_fc = r.order != SNLM_RC ? take(img) : 0;
        const size_t o_frc = (r.order == SNLM_AVG || sure) ? take(img) : 0;
        const size_t o_d1 = sure ? take(img) : 0;
        const size_t o_d2 = sure ? take(img) : 0;
        const int n_rc = (int)pass_ctas(r.W, r.H, r.S), n_cr = (int)pass_ctas(r.H, r.W, r.S);
        const size_t o_prc = sure ? take((size_t)n_rc * kPartials * sizeof(double)) : 0;
        const size_t o_pcr = sure ? take((size_t)n_cr * kPartials * sizeof(double)) : 0;
        const size_t o_info = sure ? take(16 * sizeof(double)) : 0;

        auto add_job = [&](int level, const BatchJob &j) {
            protos.push_back(Proto{j, level, i});
            return (int)protos.size() - 1;
        };
        auto rel = [&](int job, int field, size_t o) { relocs.push_back(Reloc{job, field, o}); };
        BatchJob base;
        memset(&base, 0, sizeof(base));
        base.kind = kKindPass;
        base.dep0 = base.dep1 = -1;
        const Lines img_rows = image_lines(r.img, r.dtype, r.pitch, 0);
        const Lines img_cols = image_lines(r.img, r.dtype, r.pitch, 1);
        const Lines scratch_cols{nullptr, DT_F32, 1, (long long)r.W};   // pointer relocated
        const Lines scratch_rows{nullptr, DT_F32, (long long)r.W, 1};
        int jB = -1, jD = -1;
        if (r.order != SNLM_CR) {
            BatchJob a = base;   // rows of f -> f_r (delta_1)
            a.a = pass_args(0, r.H, r.W, img_rows, nullptr, r.S, r.K, r.h, r.profile, bt);
            a.dm = dm_img;
            a.sure = sure;
            a.n_units = (int)pass_ctas(r.H, r.W, r.S);
            const int jA = add_job(0, a);
            rel(jA, R_DST, o_fr);
            if (sure)
                rel(jA, R_DOUT, o_d1);
            BatchJob b = base;   // columns of f_r -> f_rc (or out)
            b.a = pass_args(1, r.H, r.W, scratch_cols, r.order == SNLM_RC ? r.out : nullptr, r.S, r.K, r.h,
                            r.profile, bt);
            b.dm = dm_f32;
            b.sure = sure;
            b.n_units = n_rc;
            b.dep0 = jA;
            jB = add_job(1, b);
            rel(jB, R_SRC, o_fr);
            if (r.order != SNLM_RC)
                rel(jB, R_DST, o_frc);
            if (sure) {
                rel(jB, R_DIN, o_d1);
                rel(jB, R_PARTIALS, o_prc);
            }
        }
        if (r.order != SNLM_RC) {
            BatchJob c = base;   // columns of f -> f_c (delta_2)
            c.a = pass_args(1, r.H, r.W, img_cols, nullptr, r.S, r.K, r.h, r.profile, bt);
            c.dm = dm_img;
            c.sure = sure;
            c.n_units = (int)pass_ctas(r.W, r.H, r.S);
            const int jC = add_job(0, c);
            rel(jC, R_DST, o_fc);
            if (sure)
                rel(jC, R_DOUT, o_d2);
            BatchJob d = base;   // rows of f_c -> out (f_cr, or the average)
            d.a = pass_args(0, r.H, r.W, scratch_rows, r.out, r.S, r.K, r.h, r.profile, bt);
            d.dm = dm_f32;
            d.sure = sure;
            d.n_units = n_cr;
            d.dep0 = jC;
            int level = 1;
            if (r.order == SNLM_AVG || sure) {
                d.dep1 = jB;
                level = 2;
            }
            if (sure) {
                d.a.aux_f = img_rows;
                d.a.aux_rc = scratch_rows;
            }
            jD = add_job(level, d);
            rel(jD, R_SRC, o_fc);
            if (r.order == SNLM_AVG)
                rel(jD, R_BLEND, o_frc);
            if (sure) {
                rel(jD, R_DIN, o_d2);
                rel(jD, R_PARTIALS, o_pcr);
                rel(jD, R_AUXRC, o_frc);
            }
        }
        if (sure) {
            BatchJob s = base;   // the 2x2 solve of this image
            s.kind = kKindSolve;
            s.n_units = 1;
            s.dep0 = jB;
            s.dep1 = jD;
            s.n_rc = n_rc;
            s.n_cr = n_cr;
            s.sigma2 = (double)r.sigma * r.sigma;
            const int jS = add_job(3, s);
            rel(jS, R_PART_RC, o_prc);
            rel(jS, R_PART_CR, o_pcr);
            rel(jS, R_INFO, o_info);
            BatchJob m = base;   // theta1 f_rc + theta2 f_cr, in place in out
            m.kind = kKindCombine;
            m.n_px = (long long)r.H * r.W;
            m.n_units = (int)((m.n_px + kCombineChunk - 1) / kCombineChunk);
            m.dep0 = jS;
            m.out = r.out;
            const int jM = add_job(4, m);
            rel(jM, R_FRC, o_frc);
            rel(jM, R_INFO, o_info);
        }
    }
    const size_t scratch_bytes = off;

    // Classes: one per (dependency level, pass variant, K), the solve and the
    // combination jobs in classes of their own levels; the class kernels run one after
    // another on the stream in this order, so every job a class depends on lies in an
    // earlier class, complete when the class starts. Inside a class, jobs follow the
    // queue policy.
    std::vector<int> rank(n);
    for (int k = 0; k < n; ++k)
        rank[order[k]] = k;
    auto variant_of = [](const BatchJob &j) { return j.kind == kKindPass ? j.dm * 2 + j.sure : kVariantMisc; };
    auto class_K = [&](const Proto &p) { return p.j.kind == kKindPass ? reqs[p.req].K : 0; };
    std::vector<int> idx(protos.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        const Proto &pa = protos[a], &pb = protos[b];
        if (pa.level != pb.level)
            return pa.level < pb.level;
        const int va = variant_of(pa.j), vb = variant_of(pb.j);
        if (va != vb)
            return va < vb;
        const int ka = class_K(pa), kb = class_K(pb);
        if (ka != kb)
            return ka < kb;
        return rank[pa.req] < rank[pb.req];
    });
    std::vector<int> new_index(protos.size());
    for (size_t q = 0; q < idx.size(); ++q)
        new_index[idx[q]] = (int)q;
    P->jobs.resize(protos.size());
    int cur_K = -1, cur_v = -1, cur_l = -1;
    for (size_t q = 0; q < idx.size(); ++q) {
        const Proto &pr = protos[idx[q]];
        BatchJob j = pr.j;
        if (j.dep0 >= 0)
            j.dep0 = new_index[j.dep0];
        if (j.dep1 >= 0)
            j.dep1 = new_index[j.dep1];
        const int K = reqs[pr.req].K;
        const int v = variant_of(j), cK = class_K(pr);
        if (cK != cur_K || v != cur_v || pr.level != cur_l) {
            ClassInfo ci;
            ci.K = cK;
            ci.variant = v;
            ci.j0 = (int)q;
            P->classes.push_back(ci);
            cur_K = cK;
            cur_v = v;
            cur_l = pr.level;
        }
        ClassInfo &ci = P->classes.back();
        j.unit0 = ci.n_units;
        ci.n_units += j.n_units;
        ci.nj += 1;
        size_t sm = 0;
        if (j.kind == kKindPass)
            sm = max_layout_bytes(reqs[pr.req].S, K, j.sure != 0);
        else if (j.kind == kKindSolve)
            sm = (size_t)kPartials * kWarpsPerCta * 32 * sizeof(double);
        ci.smem = std::max(ci.smem, sm);
        P->jobs[q] = j;
    }
    for (Reloc &r : relocs)
        r.job = new_index[r.job];
    P->relocs = std::move(relocs);
    for (BatchJob &j : P->jobs) {
        j.need0 = j.dep0 >= 0 ? P->jobs[j.dep0].n_units : 0;
        j.need1 = j.dep1 >= 0 ? P->jobs[j.dep1].n_units : 0;
    }
    if (P->cfg.fail_job >= 0) {
        if (P->cfg.fail_job >= (int)P->jobs.size() || P->jobs[P->cfg.fail_job].dep0 < 0)
            return SNLM_ERR_ARG;
        P->jobs[P->cfg.fail_job].need0 += 1;   // never reached: host-side fault injection
    }
    for (ClassInfo &c : P->classes) {
        c.u_off = P->units;
        P->units += c.n_units;
    }
    P->unit_recs.resize((size_t)P->units);
    for (const ClassInfo &c : P->classes)
        for (int q = c.j0; q < c.j0 + c.nj; ++q) {
            const BatchJob &J = P->jobs[q];
            for (int u = 0; u < J.n_units; ++u)
                P->unit_recs[(size_t)c.u_off + J.unit0 + u] = UnitRec{q, u, J.dep0, J.need0, J.dep1, J.need1, 0, 0};
        }

    // workspace: control block | done counters | job table | unit records | scratch
    size_t o = 0;
    P->ctl_off = o;
    o += align_up(sizeof(BatchCtl), 256);
    P->done_off = o;
    o += align_up(P->jobs.size() * sizeof(int), 256);
    P->jobs_off = o;
    o += align_up(P->jobs.size() * sizeof(BatchJob), 256);
    P->units_off = o;
    o += align_up(P->unit_recs.size() * sizeof(UnitRec), 256);
    P->scratch_off = o;
    P->ws_bytes = o + scratch_bytes;
    *plan_out = P.release();
    return SNLM_OK;
}

size_t snlm_batch_plan_workspace_bytes(const snlm_batch_plan *plan)
{
    return plan ? plan->ws_bytes : 0;
}

int snlm_batch_plan_info(const snlm_batch_plan *plan, int *jobs, int *units, int *classes)
{
    if (!plan)
        return SNLM_ERR_ARG;
    if (jobs)
        *jobs = (int)plan->jobs.size();
    if (units)
        *units = plan->units;
    if (classes)
        *classes = (int)plan->classes.size();
    return SNLM_OK;
}

int snlm_batch_plan_upload(snlm_batch_plan *P, void *workspace, size_t bytes, void *stream)
{
    if (!P || !is_device_ptr(workspace) || bytes < P->ws_bytes || ((uintptr_t)workspace & 15))
        return SNLM_ERR_ARG;
    char *base = static_cast<char *>(workspace);
    char *scratch = base + P->scratch_off;
    std::vector<BatchJob> jobs = P->jobs;
    for (const Reloc &r : P->relocs) {
        BatchJob &j = jobs[r.job];
        char *p = scratch + r.offset;
        switch (r.field) {
        case R_SRC: j.a.src.ptr = p; break;
        case R_DST: j.a.dst = reinterpret_cast<float *>(p); break;
        case R_BLEND: j.a.blend = reinterpret_cast<const float *>(p); break;
        case R_DIN: j.a.delta_in = reinterpret_cast<const float *>(p); break;
        case R_DOUT: j.a.delta_out = reinterpret_cast<float *>(p); break;
        case R_PARTIALS: j.a.partials = reinterpret_cast<double *>(p); break;
        case R_AUXRC: j.a.aux_rc.ptr = p; break;
        case R_PART_RC: j.part_rc = reinterpret_cast<const double *>(p); break;
        case R_PART_CR: j.part_cr = reinterpret_cast<const double *>(p); break;
        case R_INFO: j.info = reinterpret_cast<double *>(p); break;
        case R_FRC: j.frc = reinterpret_cast<const float *>(p); break;
        default: return SNLM_ERR_ARG;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // from pageable memory the runtime stages the source before cudaMemcpyAsync
    // returns, so the local table may go out of scope right after
    cudaError_t e = cudaMemcpyAsync(base + P->jobs_off, jobs.data(), jobs.size() * sizeof(BatchJob),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !P->unit_recs.empty())
        e = cudaMemcpyAsync(base + P->units_off, P->unit_recs.data(), P->unit_recs.size() * sizeof(UnitRec),
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return status_of(e);
    // kernel attributes, one CTA per unit; a cap on CTAs per SM is applied by giving
    // each CTA that share of the SM's shared memory
    int dev = 0, smem_sm = 0, reserved = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (ClassInfo &c : P->classes) {
        BatchFn fn = batch_fn(c.K, c.variant);
        if (!fn)
            return SNLM_ERR_UNSUPPORTED;
        int occ = 0;
        e = class_occupancy(fn, dev, c.smem, &occ);
        if (e != cudaSuccess || occ < 1)
            return e != cudaSuccess ? status_of(e) : SNLM_ERR_UNSUPPORTED;
        c.smem_launch = c.smem;
        if (P->cfg.ctas_per_sm > 0 && P->cfg.ctas_per_sm < occ) {
            // the CTA's dynamic share: its part of the SM less the reserved and static
            // shared memory, and at most what one CTA may have
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, fn);
            if (e != cudaSuccess)
                return status_of(e);
            const long long st_b = (long long)fa.sharedSizeBytes;
            long long share = std::min((long long)smem_sm / P->cfg.ctas_per_sm - reserved - st_b,
                                       (long long)optin - st_b);
            share = std::max(0LL, share) & ~127LL;
            c.smem_launch = std::max(c.smem, (size_t)share);
            e = class_occupancy(fn, dev, c.smem_launch, &occ);
            if (e != cudaSuccess)
                return status_of(e);
        }
        c.grid = std::max(1, c.n_units);
    }
    P->ws = workspace;
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    if (P->graph) {
        cudaGraphDestroy(P->graph);
        P->graph = nullptr;
    }
    return SNLM_OK;
}

static int launch_raw(snlm_batch_plan *P, cudaStream_t st)
{
    char *base = static_cast<char *>(P->ws);
    BatchCtl *ctl = reinterpret_cast<BatchCtl *>(base + P->ctl_off);
    int *done = reinterpret_cast<int *>(base + P->done_off);
    const BatchJob *jobs = reinterpret_cast<const BatchJob *>(base + P->jobs_off);
    cudaError_t e = cudaMemsetAsync(base, 0, P->jobs_off, st);   // control block and counters
    if (e != cudaSuccess)
        return status_of(e);
    const unsigned long long limit_ns =
        (unsigned long long)(P->cfg.spin_limit_us > 0 ? P->cfg.spin_limit_us : 2000000) * 1000ULL;
    for (int ci = 0; ci < (int)P->classes.size(); ++ci) {
        const ClassInfo &c = P->classes[ci];
        if (c.n_units < 1)
            continue;
        TraceScope ts(SNLM_K_BATCH, st);
        const UnitRec *recs = reinterpret_cast<const UnitRec *>(base + P->units_off) + c.u_off;
        batch_fn(c.K, c.variant)<<<c.grid, kWarpsPerCta * 32, c.smem_launch, st>>>(jobs, recs, ctl, done, limit_ns);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return status_of(e);
    }
    return SNLM_OK;
}

int snlm_batch_plan_launch(snlm_batch_plan *P, void *stream)
{
    if (!P || !P->ws)
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P->exec)
        return status_of(cudaGraphLaunch(P->exec, st));
    return launch_raw(P, st);
}

int snlm_batch_plan_capture(snlm_batch_plan *P, void *stream)
{
    if (!P || !P->ws)
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!st)
        return SNLM_ERR_ARG;   // the legacy default stream cannot be captured
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    if (P->graph) {
        cudaGraphDestroy(P->graph);
        P->graph = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return status_of(e);
    const int rc = launch_raw(P, st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (rc != SNLM_OK || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != SNLM_OK ? rc : status_of(e);
    }
    e = cudaGraphInstantiate(&P->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return status_of(e);
    }
    P->graph = g;
    return SNLM_OK;
}

int snlm_batch_plan_status(snlm_batch_plan *P, void *stream)
{
    if (!P || !P->ws)
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchCtl ctl;
    cudaError_t e = cudaMemcpyAsync(&ctl, static_cast<char *>(P->ws) + P->ctl_off, sizeof(ctl),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return status_of(e);
    return ctl.err ? SNLM_ERR_TIMEOUT : SNLM_OK;
}

int snlm_batch_plan_status_async(snlm_batch_plan *P, int *host_word, void *stream)
{
    if (!P || !P->ws || !host_word)
        return SNLM_ERR_ARG;
    const size_t off = P->ctl_off + offsetof(BatchCtl, err);
    return status_of(cudaMemcpyAsync(host_word, static_cast<char *>(P->ws) + off, sizeof(int),
                                     cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
}

void snlm_batch_plan_destroy(snlm_batch_plan *P)
{
    if (!P)
        return;
    if (P->exec)
        cudaGraphExecDestroy(P->exec);
    if (P->graph)
        cudaGraphDestroy(P->graph);
    delete P;
}

}  // extern "C"
