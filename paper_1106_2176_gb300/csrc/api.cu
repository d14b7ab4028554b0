// C ABI of the GB300 FMM (include/fmm.h): handle life cycle, argument checks,
// and the order of the stages. Every numerical step runs in the kernels of
// tree.cu, expansions.cu, m2l_tc.cu and p2p.cu; nothing here computes on the
// host except the level-independent operator tables made at create time.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "fmm_internal.cuh"

namespace fmm {

static thread_local std::string tl_error;
void set_error(const std::string &msg) { tl_error = msg; }
const std::string &get_error() { return tl_error; }

void DevBuf::ensure(size_t bytes)
{
    if (bytes <= cap && p) return;
    release();
    size_t want = bytes ? bytes : 16;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        cap = 0;
        cudaGetLastError();
        throw Error{FMM_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed"};
    }
    cap = want;
}

void DevBuf::ensure_keep(size_t bytes, size_t used, cudaStream_t s)
{
    if (bytes <= cap && p) return;
    void *np = nullptr;
    size_t want = bytes ? bytes : 16;
    cudaError_t e = cudaMalloc(&np, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{FMM_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed"};
    }
    if (p && used) {
        FMM_CUDA_TRY(cudaMemcpyAsync(np, p, std::min(used, cap), cudaMemcpyDeviceToDevice, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    release();
    p = np;
    cap = want;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

void ensure_smem(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &have = set[std::make_pair(kernel, dev)];
    if (bytes <= have) return;
    FMM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
}

void PinnedBuf::ensure(size_t bytes)
{
    if (bytes <= cap && p) return;
    release();
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        throw Error{FMM_ENOMEM, "cudaMallocHost failed"};
    }
    cap = bytes;
}

void PinnedBuf::release()
{
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
}

}  // namespace fmm

fmm_ctx::~fmm_ctx()
{
    fmm::DevBuf *bufs[] = {&st_dev, &rtab64, &rtab32, &m2m_mat, &l2l_mat, &ttab, &box, &x_in, &q_in, &w_in, &keys, &keys2, &idx, &inv, &pcell, &cgeo, &energy_buf,
                           &idx2, &hist, &scan_tmp, &xs64, &xs32, &xs32lo, &c_level, &c_anchor, &c_begin, &c_end, &c_child,
                           &c_nchild, &c_parent, &c_xyz, &split_cnt, &split_off, &split_bnd, &leaves, &frontA,
                           &frontB, &p2p_pairs, &m2lx_pairs, &near_dev, &pair_keys, &pair_keys2, &pair_vals, &pair_vals2,
                           &p2p_ptr, &p2p_src, &p2p_runs, &p2p_nrun, &pr_pad, &pr_flag, &pr_pairs, &p2p_runs_pr, &m2lx_ptr, &m2lx_src, &row_cnt, &counters, &lvl_desc, &map_pool, &hash_pool,
                           &m2l_tgt, &m2l_tiles, &m2l_misc, &msplit, &Mexp, &Lexp, &far, &near, &out_phi, &out_grad,
                           &direct_part, &rot_tab, &mlat, &lat_maps};
    for (auto *b : bufs) b->release();
    hpin.release();
    lat_host.release();
    for (auto &t : tms)
        for (auto &e : t.ev)
            if (e) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (s2) cudaStreamDestroy(s2);
    if (sfar) cudaStreamDestroy(sfar);
    if (ev_far) cudaEventDestroy(ev_far);
}

using fmm::Error;

#define API_BEGIN try {
#define API_END                                   \
    }                                             \
    catch (const Error &e)                        \
    {                                             \
        fmm::set_error(e.msg);                    \
        return e.code;                            \
    }                                             \
    catch (const std::bad_alloc &)                \
    {                                             \
        fmm::set_error("host allocation failed"); \
        return FMM_ENOMEM;                        \
    }                                             \
    catch (...)                                   \
    {                                             \
        fmm::set_error("unexpected error");       \
        return FMM_ECUDA;                         \
    }

static int fail(int code, const char *msg)
{
    fmm::set_error(msg);
    return code;
}

// events of timing slot k (all slots are created with the handle, so that no
// event is created while a caller's stream is being captured)
static cudaEvent_t *slot_events(fmm_ctx *h, int64_t k) { return h->tms[k % FMM_TIMING_SLOTS].ev; }

static float ev_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

// phase times of the last k builds and evaluations, averaged (the events of
// each call are in the timing slot of its sequence number)
static void phase_means(fmm_ctx *h, int k, fmm_stats *out)
{
    out->ms_build = out->ms_evaluate = out->ms_p2m = out->ms_m2m = out->ms_m2l = 0;
    out->ms_l2l = out->ms_l2p = out->ms_p2p = out->ms_combine = 0;
    if (h->built && h->nbuilds >= k)
        for (int64_t i = h->nbuilds - k; i < h->nbuilds; i++) {
            cudaEvent_t *ev = h->tms[i % FMM_TIMING_SLOTS].ev;
            out->ms_build += ev_ms(ev[0], ev[1]) / k;
        }
    if (h->evaluated && h->nevals >= k)
        for (int64_t i = h->nevals - k; i < h->nevals; i++) {
            cudaEvent_t *ev = h->tms[i % FMM_TIMING_SLOTS].ev;
            out->ms_evaluate += ev_ms(ev[8], ev[12]) / k;
            out->ms_p2m += ev_ms(ev[2], ev[3]) / k;
            out->ms_m2m += ev_ms(ev[3], ev[4]) / k;
            out->ms_m2l += ev_ms(ev[4], ev[5]) / k;
            out->ms_l2l += ev_ms(ev[5], ev[6]) / k;
            out->ms_l2p += ev_ms(ev[6], ev[7]) / k;
            out->ms_p2p += ev_ms(ev[9], ev[10]) / k;
            out->ms_combine += ev_ms(ev[11], ev[12]) / k;
        }
}

extern "C" {

int fmm_create(int64_t N, int p, double theta, int ncrit, fmm_handle *out)
{
    if (!out) return fail(FMM_EINVAL, "fmm_create: out is NULL");
    *out = nullptr;
    if (N < 1 || N > 0x7fffffffLL) return fail(FMM_EINVAL, "fmm_create: N must be in [1, 2^31)");
    if (p < 1 || p > FMM_MAXP) return fail(FMM_EINVAL, "fmm_create: p must be in [1, 20]");
    if (!(theta > 0.0 && theta < 1.0)) return fail(FMM_EINVAL, "fmm_create: theta must be in (0, 1)");
    if (ncrit < 1) return fail(FMM_EINVAL, "fmm_create: ncrit must be >= 1");
    fmm_ctx *h = nullptr;
    API_BEGIN
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(FMM_ENODEV, "fmm_create: no CUDA device");
    }
    cudaDeviceProp prop;
    FMM_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10) return fail(FMM_ENODEV, "fmm_create: the library is built for sm_103 (Blackwell) only");
    h = new fmm_ctx();
    h->dev = dev;
    h->nsm = prop.multiProcessorCount;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    h->Nmax = N;
    h->p = p;
    h->theta = theta;
    h->cmac = theta * theta;
    h->ncrit = ncrit;
    // P2P (the compute-bound near field) runs at the lowest stream priority and
    // the far-field chain at the highest, so that the short far-field kernels
    // get SMs as soon as P2P blocks retire instead of waiting behind all of them
    int prio_lo = 0, prio_hi = 0;
    FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&h->s2, cudaStreamNonBlocking, prio_lo));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&h->sfar, cudaStreamNonBlocking, prio_hi));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_far, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    for (auto &t : h->tms)
        for (auto &e : t.ev) FMM_CUDA_TRY(cudaEventCreate(&e));
    fmm::operators_init(h);
    fmm::tensor_tables_init(h);
    FMM_CUDA_TRY(cudaDeviceSynchronize());
    *out = h;
    return FMM_OK;
    }
    catch (const Error &e)
    {
        delete h;
        fmm::set_error(e.msg);
        return e.code;
    }
    catch (...)
    {
        delete h;
        fmm::set_error("fmm_create: unexpected error");
        return FMM_ENOMEM;
    }
}

int fmm_destroy(fmm_handle h)
{
    if (!h) return fail(FMM_EINVAL, "fmm_destroy: NULL handle");
    cudaStreamSynchronize(h->stream);
    delete h;
    return FMM_OK;
}

const char *fmm_last_error(fmm_handle) { return fmm::get_error().c_str(); }

int fmm_set_precision(fmm_handle h, int mode)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_precision: NULL handle");
    if (mode != FMM_FP64 && mode != FMM_MIXED) return fail(FMM_EINVAL, "fmm_set_precision: unknown mode");
    h->precision_req = mode;
    return FMM_OK;
}

int fmm_set_m2l_engine(fmm_handle h, int engine)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_m2l_engine: NULL handle");
    if (engine != FMM_M2L_AUTO && engine != FMM_M2L_TENSOR && engine != FMM_M2L_CUDACORE && engine != FMM_M2L_ROTATION)
        return fail(FMM_EINVAL, "fmm_set_m2l_engine: unknown engine");
    if (engine == FMM_M2L_TENSOR && !fmm::tensor_m2l_supported(h))
        return fail(FMM_EINVAL, "fmm_set_m2l_engine: tensor-core M2L not supported for this p");
    if (engine == FMM_M2L_ROTATION && !fmm::rotation_m2l_supported(h))
        return fail(FMM_EINVAL, "fmm_set_m2l_engine: rotation M2L supports p <= 16");
    h->engine_req = engine;
    return FMM_OK;
}

int fmm_set_overlap(fmm_handle h, int on)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_overlap: NULL handle");
    if (on != 0 && on != 1) return fail(FMM_EINVAL, "fmm_set_overlap: on must be 0 or 1");
    h->overlap = on;
    return FMM_OK;
}

int fmm_m2l_rotation_host(int p, const double *u, const double *M, double *L)
{
    if (p < 1 || p > FMM_MAXP) return fail(FMM_EINVAL, "fmm_m2l_rotation_host: p must be in [1, 20]");
    if (!u || !M || !L) return fail(FMM_EINVAL, "fmm_m2l_rotation_host: NULL argument");
    if (!(u[0] * u[0] + u[1] * u[1] + u[2] * u[2] > 0)) return fail(FMM_EINVAL, "fmm_m2l_rotation_host: u = 0");
    try {
        fmm::m2l_rotation_ref(p, u, M, L);
    } catch (...) {
        return fail(FMM_ENOMEM, "fmm_m2l_rotation_host: out of host memory");
    }
    return FMM_OK;
}

int fmm_set_uniform_path(fmm_handle h, int on)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_uniform_path: NULL handle");
    if (on != 0 && on != 1) return fail(FMM_EINVAL, "fmm_set_uniform_path: on must be 0 or 1");
    h->uniform_req = on != 0;
    return FMM_OK;
}

int fmm_set_m2l_pool(fmm_handle h, int max_cells)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_m2l_pool: NULL handle");
    if (max_cells < -1) return fail(FMM_EINVAL, "fmm_set_m2l_pool: max_cells must be >= -1");
    h->m2l_pool = max_cells;
    return FMM_OK;
}

int fmm_set_m2l_lattice(fmm_handle h, int on)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_m2l_lattice: NULL handle");
    if (on != 0 && on != 1) return fail(FMM_EINVAL, "fmm_set_m2l_lattice: on must be 0 or 1");
    h->lattice_req = on != 0;
    return FMM_OK;
}

int fmm_set_stream(fmm_handle h, void *stream)
{
    if (!h) return fail(FMM_EINVAL, "fmm_set_stream: NULL handle");
    h->stream = (cudaStream_t)stream;
    return FMM_OK;
}

int fmm_build(fmm_handle h, const void *x, const void *q, int64_t n, int dtype)
{
    if (!h) return fail(FMM_EINVAL, "fmm_build: NULL handle");
    if (!x || !q) return fail(FMM_EINVAL, "fmm_build: NULL x or q");
    const bool host = (dtype & FMM_HOST_MEM) != 0;
    const int dt = dtype & ~FMM_HOST_MEM;
    if (dt != FMM_F32 && dt != FMM_F64) return fail(FMM_EINVAL, "fmm_build: dtype must be FMM_F32 or FMM_F64");
    if (n < 1 || n > h->Nmax) return fail(FMM_EINVAL, "fmm_build: n must be in [1, N]");
    API_BEGIN
    h->built = false;
    h->evaluated = false;
    cudaStream_t s = h->stream;
    h->n = n;
    h->dtype = dt;
    h->host_mem = host;
    h->precision = h->precision_req;
    // automatic choice: the tensor cores for the mixed path where they apply,
    // otherwise rotation (O(p^3), p <= 16), otherwise the dense CUDA-core path
    const bool tc = h->precision == FMM_MIXED && fmm::tensor_m2l_supported(h);
    if (h->engine_req == FMM_M2L_ROTATION) h->engine_used = FMM_M2L_ROTATION;
    else if (h->engine_req == FMM_M2L_CUDACORE) h->engine_used = FMM_M2L_CUDACORE;
    else if (tc) h->engine_used = FMM_M2L_TENSOR;
    else if (h->engine_req == FMM_M2L_AUTO && fmm::rotation_m2l_supported(h)) h->engine_used = FMM_M2L_ROTATION;
    else h->engine_used = FMM_M2L_CUDACORE;
    cudaEvent_t *ev = slot_events(h, h->nbuilds);
    FMM_CUDA_TRY(cudaEventRecord(ev[0], s));
    const size_t es = dt == FMM_F64 ? 8 : 4;
    const void *xd = x, *qd = q;
    if (host) {
        h->x_in.ensure(es * 3 * (size_t)n);
        h->q_in.ensure(es * (size_t)n);
        FMM_CUDA_TRY(cudaMemcpyAsync(h->x_in.p, x, es * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(h->q_in.p, q, es * (size_t)n, cudaMemcpyHostToDevice, s));
        xd = h->x_in.p;
        qd = h->q_in.p;
    }
    fmm::tree_build(h, xd, qd, n, dt);
    FMM_CUDA_TRY(cudaEventRecord(ev[1], s));
    h->nbuilds++;
    h->built = true;
    return FMM_OK;
    API_END
}

int fmm_evaluate(fmm_handle h, void *phi, void *grad)
{
    if (!h) return fail(FMM_EINVAL, "fmm_evaluate: NULL handle");
    if (!h->built) return fail(FMM_ESTATE, "fmm_evaluate: no successful fmm_build");
    if (!phi) return fail(FMM_EINVAL, "fmm_evaluate: NULL phi");
    API_BEGIN
    cudaStream_t s = h->stream;
    cudaEvent_t *ev = slot_events(h, h->nevals);
    h->ev_cur = ev;
    FMM_CUDA_TRY(cudaEventRecord(ev[8], s));
    if (h->overlap) {
        // near field and far field on two private streams, joined back to the
        // caller's stream before the combine
        FMM_CUDA_TRY(cudaEventRecord(h->ev_fork, s));
        FMM_CUDA_TRY(cudaStreamWaitEvent(h->s2, h->ev_fork, 0));
        FMM_CUDA_TRY(cudaStreamWaitEvent(h->sfar, h->ev_fork, 0));
        h->work = h->sfar;
        fmm::far_field(h);
        FMM_CUDA_TRY(cudaEventRecord(h->ev_far, h->sfar));
        FMM_CUDA_TRY(cudaEventRecord(ev[9], h->s2));
        fmm::near_field(h, h->s2);
        FMM_CUDA_TRY(cudaEventRecord(ev[10], h->s2));
        FMM_CUDA_TRY(cudaEventRecord(h->ev_join, h->s2));
        h->work = h->stream;
        FMM_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
        FMM_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_far, 0));
    } else {
        // in turn on the caller's stream
        h->work = s;
        fmm::far_field(h);
        FMM_CUDA_TRY(cudaEventRecord(ev[9], s));
        fmm::near_field(h, s);
        FMM_CUDA_TRY(cudaEventRecord(ev[10], s));
    }
    FMM_CUDA_TRY(cudaEventRecord(ev[11], s));
    const size_t es = h->dtype == FMM_F64 ? 8 : 4;
    void *pd = phi, *gd = grad;
    if (h->host_mem) {
        h->out_phi.ensure(es * (size_t)h->n);
        h->out_grad.ensure(es * 3 * (size_t)h->n);
        pd = h->out_phi.p;
        gd = h->out_grad.p;
    }
    fmm::combine_unsort(h, pd, gd);
    if (h->host_mem) {
        FMM_CUDA_TRY(cudaMemcpyAsync(phi, pd, es * (size_t)h->n, cudaMemcpyDeviceToHost, s));
        if (grad) FMM_CUDA_TRY(cudaMemcpyAsync(grad, gd, es * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, s));
    }
    FMM_CUDA_TRY(cudaEventRecord(ev[12], s));
    if (h->host_mem) FMM_CUDA_TRY(cudaStreamSynchronize(s));
    h->nevals++;
    h->evaluated = true;
    return FMM_OK;
    API_END
}

int fmm_update_charges(fmm_handle h, const void *q, const void *w)
{
    if (!h) return fail(FMM_EINVAL, "fmm_update_charges: NULL handle");
    if (!h->built) return fail(FMM_ESTATE, "fmm_update_charges: no successful fmm_build");
    if (!q) return fail(FMM_EINVAL, "fmm_update_charges: NULL q");
    API_BEGIN
    const void *qd = q, *wd = w;
    if (h->host_mem) {
        const size_t es = h->dtype == FMM_F64 ? 8 : 4;
        h->q_in.ensure(es * (size_t)h->n);
        FMM_CUDA_TRY(cudaMemcpyAsync(h->q_in.p, q, es * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
        qd = h->q_in.p;
        if (w) {
            h->w_in.ensure(es * (size_t)h->n);
            FMM_CUDA_TRY(cudaMemcpyAsync(h->w_in.p, w, es * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
            wd = h->w_in.p;
        }
    }
    fmm::update_charges(h, qd, wd);
    h->evaluated = false;
    return FMM_OK;
    API_END
}

int fmm_energy(fmm_handle h, const void *w, const void *q, const void *phi, double *out)
{
    if (!h) return fail(FMM_EINVAL, "fmm_energy: NULL handle");
    if (!h->built) return fail(FMM_ESTATE, "fmm_energy: no successful fmm_build");
    if (!w || !q || !phi || !out) return fail(FMM_EINVAL, "fmm_energy: NULL argument");
    if (h->host_mem) return fail(FMM_EINVAL, "fmm_energy: device arrays only");
    API_BEGIN
    *out = fmm::energy(h, w, q, phi);
    return FMM_OK;
    API_END
}

int fmm_energy_adjoint(fmm_handle h, double gE, const void *w, const void *q, const void *phi, const void *grad,
                       const void *psi, const void *gpsi, void *dq, void *dx, void *dw)
{
    if (!h) return fail(FMM_EINVAL, "fmm_energy_adjoint: NULL handle");
    if (!h->built) return fail(FMM_ESTATE, "fmm_energy_adjoint: no successful fmm_build");
    if (!w || !q || !phi || !psi) return fail(FMM_EINVAL, "fmm_energy_adjoint: NULL input");
    if (dx && (!grad || !gpsi)) return fail(FMM_EINVAL, "fmm_energy_adjoint: dx needs grad and gpsi");
    if (h->host_mem) return fail(FMM_EINVAL, "fmm_energy_adjoint: device arrays only");
    API_BEGIN
    fmm::energy_adjoint(h, gE, w, q, phi, grad, psi, gpsi, dq, dx, dw);
    return FMM_OK;
    API_END
}

int fmm_get_stats(fmm_handle h, fmm_stats *out)
{
    if (!h || !out) return fail(FMM_EINVAL, "fmm_get_stats: NULL argument");
    API_BEGIN
    FMM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    FMM_CUDA_TRY(cudaStreamSynchronize(h->s2));
    FMM_CUDA_TRY(cudaStreamSynchronize(h->sfar));
    std::memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->ncells = h->ncells;
    out->nleaves = h->nleaves;
    out->depth = h->depth;
    out->precision = h->precision;
    out->n_p2p_pairs = h->n_p2p;
    out->n_m2l_pairs = fmm::tree_m2l_total(h);
    out->n_m2l_irregular = h->n_m2lx;
    out->n_interactions = h->n_interactions;
    out->n_stencil = h->st_off.empty() ? 0 : h->st_off[8];
    out->m2l_engine = h->engine_used;
    if (h->m2l_misc.p) {
        // device-side timeouts of the last evaluate: M2L (bit 0), P2P (bit 1)
        int e[2] = {0, 0};
        FMM_CUDA_TRY(cudaMemcpy(e, h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1) + 4, sizeof(e),
                                cudaMemcpyDeviceToHost));
        out->async_error = (e[0] ? 1 : 0) | (e[1] ? 2 : 0);
    }
    out->kernel_launches = h->launches;
    out->uniform_path = h->uniform_used ? 1 : 0;
    out->lattice_levels = (int32_t)h->lat_levels;
    phase_means(h, 1, out);
    return FMM_OK;
    API_END
}

int fmm_get_stats_mean(fmm_handle h, int k, fmm_stats *out)
{
    if (!h || !out) return fail(FMM_EINVAL, "fmm_get_stats_mean: NULL argument");
    if (k < 1 || k > FMM_TIMING_SLOTS || k > h->nbuilds || k > h->nevals)
        return fail(FMM_EINVAL, "fmm_get_stats_mean: k must be in [1, 32] and at most the builds and evaluations done");
    const int rc = fmm_get_stats(h, out);
    if (rc != FMM_OK) return rc;
    API_BEGIN
    phase_means(h, k, out);
    return FMM_OK;
    API_END
}

int fmm_get_tree_sizes(fmm_handle h, fmm_tree_sizes *out)
{
    if (!h || !out) return fail(FMM_EINVAL, "fmm_get_tree_sizes: NULL argument");
    if (!h->built) return fail(FMM_ESTATE, "fmm_get_tree_sizes: no successful fmm_build");
    out->n = h->n;
    out->ncells = h->ncells;
    out->n_p2p = h->n_p2p;
    out->n_m2l = fmm::tree_m2l_total(h);
    out->depth = h->depth;
    out->p = h->p;
    return FMM_OK;
}

int fmm_export_tree(fmm_handle h, uint64_t *keys, int32_t *perm, int32_t *level, uint64_t *anchor, int32_t *begin,
                    int32_t *end, int32_t *child, int32_t *nchild, int32_t *parent, int64_t *p2p_ptr, int32_t *p2p_idx,
                    int64_t *m2l_ptr, int32_t *m2l_idx, double *box)
{
    if (!h) return fail(FMM_EINVAL, "fmm_export_tree: NULL handle");
    if (!h->built) return fail(FMM_ESTATE, "fmm_export_tree: no successful fmm_build");
    API_BEGIN
    fmm::tree_export(h, keys, perm, level, anchor, begin, end, child, nchild, parent, p2p_ptr, p2p_idx, m2l_ptr,
                     m2l_idx, box);
    return FMM_OK;
    API_END
}

int fmm_export_expansions(fmm_handle h, double *M, double *L)
{
    if (!h) return fail(FMM_EINVAL, "fmm_export_expansions: NULL handle");
    if (!h->evaluated) return fail(FMM_ESTATE, "fmm_export_expansions: no successful fmm_evaluate");
    API_BEGIN
    const size_t cnt = (size_t)h->ncells * h->p * h->p;
    FMM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 2; k++) {
        double *dst = k ? L : M;
        if (!dst) continue;
        const fmm::DevBuf &src = k ? h->Lexp : h->Mexp;
        if (h->precision == FMM_FP64) {
            FMM_CUDA_TRY(cudaMemcpy(dst, src.p, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> tmp(cnt);
            FMM_CUDA_TRY(cudaMemcpy(tmp.data(), src.p, sizeof(float) * cnt, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < cnt; i++) dst[i] = tmp[i];
        }
    }
    return FMM_OK;
    API_END
}

int fmm_direct(fmm_handle h, const double *x, const double *q, int64_t n, const int64_t *tidx, int64_t nt, double *phi,
               double *grad)
{
    if (!h) return fail(FMM_EINVAL, "fmm_direct: NULL handle");
    if (!x || !q || !phi) return fail(FMM_EINVAL, "fmm_direct: NULL pointer");
    if (n < 1 || nt < 1 || (tidx == nullptr && nt != n)) return fail(FMM_EINVAL, "fmm_direct: bad sizes");
    API_BEGIN
    fmm::direct_sum(h, x, q, n, tidx, nt, phi, grad);
    return FMM_OK;
    API_END
}

}  // extern "C"
