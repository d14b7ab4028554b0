// Batched evaluation of many independent systems (fmm_batch_* in
// include/fmm.h): the paper's GPU task-queue idea (Sec. 5: work for the GPU
// queued in large, contiguous pieces) applied to many small FMMs. Each system
// keeps its own handle, tree and lists; one evaluation of the whole batch is
// a handful of launches whose blocks or warps draw work items (system, phase,
// cell or tile) from device queues:
//   zero     local expansions and dependency counters of every system
//   up       P2M of every leaf, then M2M from the deepest level up (per-warp
//            items; an M2M item waits, bounded, until the level below is done)
//   pad      multipole rows padded to whole k-blocks (tensor-core M2L)
//   M2L      same-level pairs on the tensor cores, persistent over (system, tile)
//   M2L'     pairs across levels of adaptive trees, one block per target cell
//   down     L2L from the top level down, then L2P (bounded waits per level)
//   P2P      persistent over (system, target leaf), on a second stream
//   combine  far + near back to every system's caller order
// Every item runs the arithmetic of the single-system kernels, so each
// system's result is bitwise that of its own fmm_evaluate.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

struct fmm_batch_s {
    int nsys = 0, p = 0, dev = 0, nsm = 0;
    std::vector<fmm_ctx *> hs;
    fmm::DevBuf sys, cnt, up, dn, mx, pp, jobs, blk0, misc;
    int n_up = 0, n_dn = 0, n_mx = 0, n_pp = 0, n_jobs = 0, n_blk = 0;
    std::vector<int4> up_host, dn_host;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~fmm_batch_s()
    {
        for (auto *b : {&sys, &cnt, &up, &dn, &mx, &pp, &jobs, &blk0, &misc}) b->release();
        if (side) cudaStreamDestroy(side);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    }
};

namespace fmm {

// misc: [0] up queue, [1] down queue, [2] M2L queue, [3] P2P queue,
// [4] dependency waits (bit 0), [5] tensor-core M2L, [6] P2P
enum { BQ_UP = 0, BQ_DN = 1, BQ_M2L = 2, BQ_P2P = 3, BE_DEP = 4, BE_M2L = 5, BE_P2P = 6, BMISC = 8 };

template <class T>
static void upload(DevBuf &b, const std::vector<T> &v)
{
    b.ensure(sizeof(T) * std::max<size_t>(v.size(), 1));
    if (!v.empty()) FMM_CUDA_TRY(cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
}

}  // namespace fmm

using fmm::Error;

extern "C" {

int fmm_batch_create(const fmm_handle *handles, int nsys, void *const *phi, void *const *grad, fmm_batch *out)
{
    using namespace fmm;
    if (!out) {
        set_error("fmm_batch_create: out is NULL");
        return FMM_EINVAL;
    }
    *out = nullptr;
    if (!handles || !phi || !grad || nsys < 1) {
        set_error("fmm_batch_create: NULL arrays or nsys < 1");
        return FMM_EINVAL;
    }
    fmm_batch_s *b = nullptr;
    try {
        const int p = handles[0] ? handles[0]->p : 0;
        for (int i = 0; i < nsys; i++) {
            fmm_ctx *h = handles[i];
            if (!h || !phi[i] || !grad[i]) throw Error{FMM_EINVAL, "fmm_batch_create: NULL handle or output"};
            if (!h->built) throw Error{FMM_ESTATE, "fmm_batch_create: every handle needs a successful fmm_build"};
            if (h->precision != FMM_MIXED || h->dtype != FMM_F32 || h->host_mem)
                throw Error{FMM_EINVAL, "fmm_batch_create: mixed precision, FP32 device inputs only"};
            if (h->p != p || h->dev != handles[0]->dev)
                throw Error{FMM_EINVAL, "fmm_batch_create: all systems need the same p and device"};
            if (h->engine_used != FMM_M2L_TENSOR || !h->pr_ready)
                throw Error{FMM_EINVAL, "fmm_batch_create: systems must use the tensor-core M2L (p in [2, 10])"};
        }
        if (p < 2 || p > 10) throw Error{FMM_EINVAL, "fmm_batch_create: p must be in [2, 10]"};
        b = new fmm_batch_s();
        b->nsys = nsys;
        b->p = p;
        b->dev = handles[0]->dev;
        b->nsm = handles[0]->nsm;
        b->hs.assign(handles, handles + nsys);
        FMM_CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        FMM_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        FMM_CUDA_TRY(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
        const int PP = p * p;
        b->cnt.ensure(sizeof(unsigned) * 2 * (FMM_MAXLEVEL + 1) * (size_t)nsys);
        b->misc.ensure(sizeof(int) * BMISC);
        FMM_CUDA_TRY(cudaMemset(b->misc.p, 0, sizeof(int) * BMISC));
        std::vector<BatchSys> sd((size_t)nsys);
        std::vector<M2LJob> jobs;
        std::vector<int2> mx, pp;
        std::vector<int> blk0;
        int maxdepth = 0, item0 = 0, nblk = 0;
        std::vector<std::vector<int>> nchild((size_t)nsys), leaves((size_t)nsys);
        for (int i = 0; i < nsys; i++) {
            fmm_ctx *h = handles[i];
            cudaStream_t s = h->stream;
            h->Mexp.ensure(sizeof(float) * (size_t)h->ncells * PP);
            h->Lexp.ensure(sizeof(float) * (size_t)h->ncells * PP);
            h->far.ensure(sizeof(double4_32a) * (size_t)h->n);
            h->near.ensure(sizeof(double4_32a) * (size_t)h->n);
            cell_geometry(h, s);
            BatchSys &S = sd[(size_t)i];
            std::memset(&S, 0, sizeof(S));
            S.leaves = h->leaves.as<int>();
            S.begin = h->c_begin.as<int>();
            S.end = h->c_end.as<int>();
            S.child = h->c_child.as<int>();
            S.nchild = h->c_nchild.as<int>();
            S.parent = h->c_parent.as<int>();
            S.pcell = h->pcell.as<int>();
            S.inv = h->inv.as<int>();
            S.xyz = h->c_xyz.as<int4>();
            S.box = h->box.as<Box>();
            S.cgeo = h->cgeo.as<double4_32a>();
            S.xs = h->xs32.as<float4>();
            S.M = h->Mexp.as<float>();
            S.L = h->Lexp.as<float>();
            S.far = h->far.as<double4_32a>();
            S.near = h->near.as<double4_32a>();
            S.m2lx_ptr = h->m2lx_ptr.as<int>();
            S.m2lx_src = h->m2lx_src.as<int>();
            S.pairs = h->pr_pairs.as<float>();
            S.pad = h->pr_pad.as<unsigned>();
            S.flag = h->pr_flag.as<unsigned>();
            S.p2p_ptr = h->p2p_ptr.as<int>();
            S.nrun = h->p2p_nrun.as<int>();
            S.runs_pr = h->p2p_runs_pr.as<int2>();
            S.phi = static_cast<float *>(phi[i]);
            S.grad = static_cast<float *>(grad[i]);
            S.cnt_up = b->cnt.as<unsigned>() + (size_t)i * 2 * (FMM_MAXLEVEL + 1);
            S.cnt_dn = S.cnt_up + (FMM_MAXLEVEL + 1);
            S.n = (int)h->n;
            S.ncells = h->ncells;
            S.nleaves = h->nleaves;
            S.depth = h->depth;
            for (int l = 0; l <= FMM_MAXLEVEL + 1; l++)
                S.lvl_start[l] = l < (int)h->lvl_start.size() ? h->lvl_start[(size_t)l] : h->ncells;
            S.c0 = h->depth >= 2 ? h->lvl_start[2] : h->ncells;
            maxdepth = std::max(maxdepth, h->depth);
            // same-level M2L: the system's tiles in the persistent tensor-core launch
            if (h->depth >= 2) {
                M2LJob j = m2l_tensor_job(h, S.L, S.M, s);
                if (j.mrow != S.M) S.mpad = const_cast<float *>(j.mrow);
                int nt = 0;
                FMM_CUDA_TRY(cudaMemcpy(&nt, j.ntiles, sizeof(int), cudaMemcpyDeviceToHost));
                j.item0 = item0;
                j.count = nt;
                item0 += nt;
                if (nt > 0) jobs.push_back(j);
            }
            // tree structure for the work lists
            nchild[(size_t)i].resize((size_t)h->ncells);
            leaves[(size_t)i].resize((size_t)h->nleaves);
            FMM_CUDA_TRY(cudaMemcpy(nchild[(size_t)i].data(), S.nchild, sizeof(int) * (size_t)h->ncells, cudaMemcpyDeviceToHost));
            FMM_CUDA_TRY(cudaMemcpy(leaves[(size_t)i].data(), S.leaves, sizeof(int) * (size_t)h->nleaves, cudaMemcpyDeviceToHost));
            if (h->n_m2lx > 0) {
                std::vector<int> ptr((size_t)h->ncells + 1);
                FMM_CUDA_TRY(cudaMemcpy(ptr.data(), S.m2lx_ptr, sizeof(int) * ptr.size(), cudaMemcpyDeviceToHost));
                for (int c = 0; c < h->ncells; c++)
                    if (ptr[(size_t)c + 1] > ptr[(size_t)c]) mx.push_back(make_int2(i, c));
            }
            blk0.push_back(nblk);
            nblk += (int)((h->n + 255) / 256);
        }
        // work lists in dependency order: P2M of every leaf, then M2M level by
        // level from the deepest; L2L level by level from the top, then L2P
        auto level_of = [&](int i, int c) {
            const BatchSys &S = sd[(size_t)i];
            int l = 0;
            while (l < S.depth && c >= S.lvl_start[l + 1]) l++;
            return l;
        };
        for (int i = 0; i < nsys; i++)
            for (int c : leaves[(size_t)i]) {
                b->up_host.push_back(make_int4(i, BATCH_P2M, c, level_of(i, c)));
                pp.push_back(make_int2(i, c));
            }
        for (int l = maxdepth - 1; l >= 0; l--)
            for (int i = 0; i < nsys; i++) {
                const BatchSys &S = sd[(size_t)i];
                if (l >= S.depth) continue;
                for (int c = S.lvl_start[l]; c < S.lvl_start[l + 1]; c++)
                    if (nchild[(size_t)i][(size_t)c] > 0) b->up_host.push_back(make_int4(i, BATCH_M2M, c, l));
            }
        for (int l = 1; l <= maxdepth; l++)
            for (int i = 0; i < nsys; i++) {
                const BatchSys &S = sd[(size_t)i];
                if (l > S.depth) continue;
                for (int c = S.lvl_start[l]; c < S.lvl_start[l + 1]; c++) b->dn_host.push_back(make_int4(i, BATCH_L2L, c, l));
            }
        for (int i = 0; i < nsys; i++)
            for (int c : leaves[(size_t)i]) b->dn_host.push_back(make_int4(i, BATCH_L2P, c, level_of(i, c)));
        blk0.push_back(nblk);
        upload(b->sys, sd);
        upload(b->up, b->up_host);
        upload(b->dn, b->dn_host);
        upload(b->mx, mx);
        upload(b->pp, pp);
        upload(b->jobs, jobs);
        upload(b->blk0, blk0);
        b->n_up = (int)b->up_host.size();
        b->n_dn = (int)b->dn_host.size();
        b->n_mx = (int)mx.size();
        b->n_pp = (int)pp.size();
        b->n_jobs = (int)jobs.size();
        b->n_blk = nblk;
        FMM_CUDA_TRY(cudaDeviceSynchronize());
        *out = b;
        return FMM_OK;
    } catch (const Error &e) {
        delete b;
        set_error(e.msg);
        return e.code;
    } catch (...) {
        delete b;
        set_error("fmm_batch_create: out of host memory");
        return FMM_ENOMEM;
    }
}

int fmm_batch_evaluate(fmm_batch b, void *stream)
{
    using namespace fmm;
    if (!b) {
        set_error("fmm_batch_evaluate: NULL batch");
        return FMM_EINVAL;
    }
    try {
        cudaStream_t s = (cudaStream_t)stream;
        const BatchSys *sys = b->sys.as<BatchSys>();
        int *misc = b->misc.as<int>();
        fmm_ctx *h0 = b->hs[0];
        FMM_CUDA_TRY(cudaMemsetAsync(misc + BE_DEP, 0, sizeof(int) * 3, s));
        // the near field has no dependency on the far field: second stream
        FMM_CUDA_TRY(cudaEventRecord(b->fork, s));
        FMM_CUDA_TRY(cudaStreamWaitEvent(b->side, b->fork, 0));
        batch_p2p(b->nsm, sys, b->pp.as<int2>(), b->n_pp, misc + BQ_P2P, misc + BE_P2P, b->side);
        FMM_CUDA_TRY(cudaEventRecord(b->join, b->side));
        batch_zero(b->p, sys, b->nsys, s);
        batch_up(b->p, b->nsm, sys, b->up.as<int4>(), b->n_up, misc + BQ_UP, h0->m2m_mat.as<float>(), misc + BE_DEP, s);
        batch_mpad(b->p, sys, b->nsys, s);
        if (b->n_jobs > 0)
            m2l_tensor_jobs(b->p, b->nsm, b->jobs.as<M2LJob>(), b->n_jobs, misc + BQ_M2L, misc + BE_M2L, s);
        batch_m2lx(b->p, sys, b->mx.as<int2>(), b->n_mx, s);
        batch_down(b->p, b->nsm, sys, b->dn.as<int4>(), b->n_dn, misc + BQ_DN, h0->l2l_mat.as<float>(), misc + BE_DEP, s);
        FMM_CUDA_TRY(cudaStreamWaitEvent(s, b->join, 0));
        batch_combine(sys, b->nsys, b->blk0.as<int>(), b->n_blk, s);
        return FMM_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

int fmm_batch_status(fmm_batch b, int *async_error, int64_t *kernel_launches)
{
    using namespace fmm;
    if (!b || !async_error) {
        set_error("fmm_batch_status: NULL argument");
        return FMM_EINVAL;
    }
    try {
        int e[3] = {0, 0, 0};
        FMM_CUDA_TRY(cudaDeviceSynchronize());
        FMM_CUDA_TRY(cudaMemcpy(e, b->misc.as<int>() + BE_DEP, sizeof(e), cudaMemcpyDeviceToHost));
        *async_error = (e[0] ? 1 : 0) | (e[1] ? 2 : 0) | (e[2] ? 4 : 0);
        if (kernel_launches) *kernel_launches = 6 + (b->n_mx > 0 ? 1 : 0) + (b->p * b->p % 32 != 0 ? 1 : 0);
        return FMM_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

int fmm_batch_withhold(fmm_batch b, int pass, int64_t item)
{
    using namespace fmm;
    if (!b || (pass != 0 && pass != 1)) {
        set_error("fmm_batch_withhold: NULL batch or pass not 0 (up) / 1 (down)");
        return FMM_EINVAL;
    }
    std::vector<int4> &v = pass == 0 ? b->up_host : b->dn_host;
    if (item < 0 || item >= (int64_t)v.size()) {
        set_error("fmm_batch_withhold: item out of range");
        return FMM_EINVAL;
    }
    try {
        v.erase(v.begin() + item);
        upload(pass == 0 ? b->up : b->dn, v);
        (pass == 0 ? b->n_up : b->n_dn) = (int)v.size();
        return FMM_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

int fmm_batch_items(fmm_batch b, int pass, int64_t item, int *system, int *kind, int *cell, int *level)
{
    using namespace fmm;
    if (!b || (pass != 0 && pass != 1) || !system || !kind || !cell || !level) {
        set_error("fmm_batch_items: bad argument");
        return FMM_EINVAL;
    }
    const std::vector<int4> &v = pass == 0 ? b->up_host : b->dn_host;
    if (item < 0 || item >= (int64_t)v.size()) {
        set_error("fmm_batch_items: item out of range");
        return FMM_EINVAL;
    }
    const int4 it = v[(size_t)item];
    *system = it.x;
    *kind = it.y;
    *cell = it.z;
    *level = it.w;
    return FMM_OK;
}

int fmm_batch_destroy(fmm_batch b)
{
    if (!b) {
        fmm::set_error("fmm_batch_destroy: NULL batch");
        return FMM_EINVAL;
    }
    cudaDeviceSynchronize();
    delete b;
    return FMM_OK;
}

}  // extern "C"
