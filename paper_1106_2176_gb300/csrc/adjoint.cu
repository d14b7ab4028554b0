// Charges on a built tree, the weighted energy and its adjoint.
//
// For the weighted energy E = 1/2 sum_i w_i q_i phi_i of the Laplace potential
// phi_i = sum_{j != i} q_j / r_ij, the kernel is symmetric, so
//   dE/dq_k = 1/2 (w_k phi_k + psi_k),
//   dE/dx_k = 1/2 q_k (w_k grad phi_k + grad psi_k),
//   dE/dw_k = 1/2 q_k phi_k,
// where psi is the potential of the charges w_j q_j at the same positions:
// one more FMM evaluation on the same tree (fmm_update_charges, then
// fmm_evaluate). Nothing of the first evaluation is kept but phi and grad.
#include "fmm_internal.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// new charges q (times w if given) into the sorted particle arrays
template <class T>
__global__ void charges_k(const T *__restrict__ q, const T *__restrict__ w, const int *__restrict__ idx, int64_t n,
                          double4_32a *__restrict__ xs64, float4 *__restrict__ xs32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = idx[i];
    const double c = w ? (double)q[j] * (double)w[j] : (double)q[j];
    if (xs64) xs64[i].w = c;
    if (xs32) xs32[i].w = (float)c;
}

void update_charges(fmm_ctx *h, const void *q, const void *w)
{
    cudaStream_t s = h->stream;
    double4_32a *xs64 = h->xs64.p ? h->xs64.as<double4_32a>() : nullptr;
    float4 *xs32 = (h->precision == FMM_MIXED && h->xs32.p) ? h->xs32.as<float4>() : nullptr;
    if (h->precision == FMM_FP64) xs32 = nullptr;
    if (h->dtype == FMM_F64)
        charges_k<double><<<nblk(h->n, 256), 256, 0, s>>>((const double *)q, (const double *)w, h->idx.as<int>(), h->n,
                                                           xs64, xs32);
    else
        charges_k<float><<<nblk(h->n, 256), 256, 0, s>>>((const float *)q, (const float *)w, h->idx.as<int>(), h->n,
                                                          xs64, xs32);
    count_launch(h);
    check_launch("charges");
    p2p_pairs_fill(h, s);  // the packed P2P reads the charges from its pair records
}

// E = 1/2 sum w q phi: FP64 block sums, then the blocks in order
constexpr int EN_T = 256;

template <class T>
__global__ void __launch_bounds__(EN_T) energy_k(const T *__restrict__ w, const T *__restrict__ q, const T *__restrict__ phi,
                                                 int64_t n, double *__restrict__ part)
{
    __shared__ double sh[EN_T];
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * EN_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * EN_T)
        a += (double)w[i] * (double)q[i] * (double)phi[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = EN_T / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void energy_final_k(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    double a = 0.0;
    for (int b = 0; b < nb; b++) a += part[b];
    *out = 0.5 * a;
}

double energy(fmm_ctx *h, const void *w, const void *q, const void *phi)
{
    cudaStream_t s = h->stream;
    const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (h->n + EN_T - 1) / EN_T));
    h->energy_buf.ensure(sizeof(double) * (size_t)(nb + 1));
    double *part = h->energy_buf.as<double>();
    if (h->dtype == FMM_F64)
        energy_k<double><<<nb, EN_T, 0, s>>>((const double *)w, (const double *)q, (const double *)phi, h->n, part);
    else
        energy_k<float><<<nb, EN_T, 0, s>>>((const float *)w, (const float *)q, (const float *)phi, h->n, part);
    count_launch(h);
    energy_final_k<<<1, 1, 0, s>>>(part, nb, part + nb);
    count_launch(h);
    check_launch("energy");
    double e = 0.0;
    FMM_CUDA_TRY(cudaMemcpyAsync(h->hpin.as<char>() + 4096 + 1024, part + nb, sizeof(double), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(&e, h->hpin.as<char>() + 4096 + 1024, sizeof(double));
    return e;
}

template <class T>
__global__ void adjoint_k(int64_t n, double gE, const T *__restrict__ w, const T *__restrict__ q, const T *__restrict__ phi,
                          const T *__restrict__ grad, const T *__restrict__ psi, const T *__restrict__ gpsi,
                          T *__restrict__ dq, T *__restrict__ dx, T *__restrict__ dw)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double wi = w[i], qi = q[i], f = 0.5 * gE;
    if (dq) dq[i] = (T)(f * (wi * (double)phi[i] + (double)psi[i]));
    if (dw) dw[i] = (T)(f * qi * (double)phi[i]);
    if (dx)
#pragma unroll
        for (int d = 0; d < 3; d++)
            dx[3 * i + d] = (T)(f * qi * (wi * (double)grad[3 * i + d] + (double)gpsi[3 * i + d]));
}

void energy_adjoint(fmm_ctx *h, double gE, const void *w, const void *q, const void *phi, const void *grad,
                    const void *psi, const void *gpsi, void *dq, void *dx, void *dw)
{
    cudaStream_t s = h->stream;
    if (h->dtype == FMM_F64)
        adjoint_k<double><<<nblk(h->n, 256), 256, 0, s>>>(h->n, gE, (const double *)w, (const double *)q,
                                                           (const double *)phi, (const double *)grad, (const double *)psi,
                                                           (const double *)gpsi, (double *)dq, (double *)dx, (double *)dw);
    else
        adjoint_k<float><<<nblk(h->n, 256), 256, 0, s>>>(h->n, gE, (const float *)w, (const float *)q, (const float *)phi,
                                                          (const float *)grad, (const float *)psi, (const float *)gpsi,
                                                          (float *)dq, (float *)dx, (float *)dw);
    count_launch(h);
    check_launch("energy adjoint");
}

}  // namespace fmm
