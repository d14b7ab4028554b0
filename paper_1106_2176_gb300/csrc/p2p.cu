// Near field (P2P), the FP64 direct sum and the final combine/unsort.
//
// P2P is the kernel that takes most of the FMM time (Sec. 3.1 of Yokota &
// Barba, arXiv:1106.2176) and the one their SIMD tuning targets (Sec. 3.2):
//   phi_i += sum_j q_j / r_ij,   grad_i -= sum_j q_j (x_i - x_j) / r_ij^3
// over the particles j of every leaf in the P2P list of i's leaf, skipping
// j == i and coincident pairs (r_ij = 0).
//
// GPU mapping: one block of 128 threads per target leaf. Each thread owns two
// targets (i and i + R, R = ceil(n_leaf / 2) rows) and one of S = 128 / R
// slices of the source stream, so a leaf of ~38 particles keeps ~114 of 128
// threads busy. Source leaves are concatenated into a shared-memory chunk;
// threads of one slice read the same source (broadcast), FMA and rsqrt run on
// the CUDA cores. In FP32 the sum over a slice is taken in blocks of 64
// sources whose totals are added with TwoSum, and slices are combined in FP64
// in a fixed order, so the result does not depend on scheduling.
#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <class T>
struct Vec4;
template <>
struct Vec4<float> { using type = float4; };
template <>
struct Vec4<double> { using type = double4_32a; };

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <class T, class T4>
__device__ __forceinline__ void interact(const T4 &t, const T4 &s, T &p, T &gx, T &gy, T &gz)
{
    const T dx = t.x - s.x, dy = t.y - s.y, dz = t.z - s.z;
    const T r2 = dx * dx + dy * dy + dz * dz;
    T ri = rsq(r2);
    ri = r2 > T(0) ? ri : T(0);
    const T qr = s.w * ri;
    const T qr3 = qr * ri * ri;
    p += qr;
    gx -= qr3 * dx;
    gy -= qr3 * dy;
    gz -= qr3 * dz;
}

// running sum (hi, lo) += b, error-free (TwoSum)
__device__ __forceinline__ void acc2(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += err;
}
__device__ __forceinline__ void acc2(double &hi, double &lo, double b) { hi += b; }

constexpr int P2P_T = 128;

template <class T4>
__device__ __forceinline__ void interact_ds(const T4 &t, const float4 &tl, const T4 &s, const float4 &sl, float &p, float &gx,
                                            float &gy, float &gz)
{
    const float dx = (t.x - s.x) + (tl.x - sl.x), dy = (t.y - s.y) + (tl.y - sl.y), dz = (t.z - s.z) + (tl.z - sl.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    float ri = rsqrtf(r2);
    ri = r2 > 0.f ? ri : 0.f;
    const float qr = s.w * ri;
    const float qr3 = qr * ri * ri;
    p += qr;
    gx -= qr3 * dx;
    gy -= qr3 * dy;
    gz -= qr3 * dz;
}

// DS (FP32 path, FP64 input): every coordinate is carried as an FP32 pair
// (hi, lo) and a difference is formed as (hi_i - hi_j) + (lo_i - lo_j); for
// nearby particles hi_i - hi_j is exact, so the near field keeps the accuracy
// of the FP64 positions. FP32 inputs have lo = 0 and use the plain form.
template <class T, bool DS>
__global__ void __launch_bounds__(P2P_T) p2p_k(const typename Vec4<T>::type *__restrict__ xs, const float4 *__restrict__ xlo,
                                               const int *__restrict__ leaves, const int *__restrict__ begin,
                                               const int *__restrict__ end, const int *__restrict__ ptr,
                                               const int *__restrict__ src, double4_32a *__restrict__ near)
{
    using T4 = typename Vec4<T>::type;
    constexpr int CH = (DS || sizeof(T) == 8) ? 1024 : 2048;
    __shared__ T4 sh[CH];
    __shared__ float4 shlo[DS ? CH : 1];
    __shared__ double red[P2P_T * 8];
    const int A = leaves[blockIdx.x];
    const int tb = begin[A], te = end[A];
    const int k0 = ptr[A], k1 = ptr[A + 1];
    for (int t0 = tb; t0 < te; t0 += 2 * P2P_T) {
        const int nt = min(2 * P2P_T, te - t0);
        const int R = (nt + 1) >> 1;
        const int S = max(1, P2P_T / R);
        const int row = threadIdx.x % R, sl = threadIdx.x / R;
        const bool act = sl < S;
        const bool has1 = act && (row + R < nt);
        T4 x0 = {}, x1 = {};
        float4 l0 = {}, l1 = {};
        if (act) {
            x0 = xs[t0 + row];
            if (DS) l0 = xlo[t0 + row];
        }
        x1 = has1 ? xs[t0 + row + R] : x0;
        if (DS) l1 = has1 ? xlo[t0 + row + R] : l0;
        T h[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lo[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int k = k0, off = 0;
        while (k < k1) {
            __syncthreads();
            int fill = 0;
            while (k < k1 && fill < CH) {
                const int B = src[k];
                const int b0 = begin[B] + off;
                const int blen = end[B] - b0;
                const int take = min(blen, CH - fill);
                for (int j = threadIdx.x; j < take; j += P2P_T) {
                    sh[fill + j] = xs[b0 + j];
                    if (DS) shlo[fill + j] = xlo[b0 + j];
                }
                fill += take;
                if (take == blen) {
                    k++;
                    off = 0;
                } else off += take;
            }
            __syncthreads();
            if (act) {
                const int jlo = (int)(((long long)fill * sl) / S), jhi = (int)(((long long)fill * (sl + 1)) / S);
                for (int j0 = jlo; j0 < jhi; j0 += 64) {
                    const int j1 = min(jhi, j0 + 64);
                    T b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
                    for (int j = j0; j < j1; j++) {
                        const T4 s = sh[j];
                        if constexpr (DS) {
                            const float4 q = shlo[j];
                            interact_ds(x0, l0, s, q, b[0], b[1], b[2], b[3]);
                            interact_ds(x1, l1, s, q, b[4], b[5], b[6], b[7]);
                        } else {
                            interact(x0, s, b[0], b[1], b[2], b[3]);
                            interact(x1, s, b[4], b[5], b[6], b[7]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 8; c++) acc2(h[c], lo[c], b[c]);
                }
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int c = 0; c < 8; c++) red[(sl * R + row) * 8 + c] = (double)h[c] + (double)lo[c];
        }
        __syncthreads();
        if ((int)threadIdx.x < R) {
            double o[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int s2 = 0; s2 < S; s2++)
#pragma unroll
                for (int c = 0; c < 8; c++) o[c] += red[(s2 * R + threadIdx.x) * 8 + c];
            near[t0 + threadIdx.x] = make_double4_32a(o[0], o[1], o[2], o[3]);
            if ((int)threadIdx.x + R < nt) near[t0 + threadIdx.x + R] = make_double4_32a(o[4], o[5], o[6], o[7]);
        }
    }
}

void near_field(fmm_ctx *h, cudaStream_t s)
{
    h->near.ensure(sizeof(double4_32a) * (size_t)h->n);
    if (h->nleaves == 0) return;
    const int *lv = h->leaves.as<int>(), *cb = h->c_begin.as<int>(), *ce = h->c_end.as<int>();
    const int *pp = h->p2p_ptr.as<int>(), *ps = h->p2p_src.as<int>();
    double4_32a *out = h->near.as<double4_32a>();
    if (h->precision == FMM_FP64)
        p2p_k<double, false><<<h->nleaves, P2P_T, 0, s>>>(h->xs64.as<double4_32a>(), nullptr, lv, cb, ce, pp, ps, out);
    else if (h->dtype == FMM_F64)
        p2p_k<float, true><<<h->nleaves, P2P_T, 0, s>>>(h->xs32.as<float4>(), h->xs32lo.as<float4>(), lv, cb, ce, pp, ps, out);
    else
        p2p_k<float, false><<<h->nleaves, P2P_T, 0, s>>>(h->xs32.as<float4>(), nullptr, lv, cb, ce, pp, ps, out);
    count_launch(h);
    check_launch("p2p");
}

// ---------------------------------------------------------------------------
// far + near, back to the caller's particle order and element type
// ---------------------------------------------------------------------------
template <class OT>
__global__ void combine_k(const double4_32a *__restrict__ far, const double4_32a *__restrict__ near, const int *__restrict__ perm,
                          int64_t n, OT *__restrict__ phi, OT *__restrict__ grad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    const double4_32a a = far[i], b = near[i];
    phi[j] = (OT)(a.x + b.x);
    if (grad) {
        grad[3 * j + 0] = (OT)(a.y + b.y);
        grad[3 * j + 1] = (OT)(a.z + b.z);
        grad[3 * j + 2] = (OT)(a.w + b.w);
    }
}

void combine_unsort(fmm_ctx *h, void *phi, void *grad)
{
    if (h->dtype == FMM_F64)
        combine_k<double><<<nblk(h->n, 256), 256, 0, h->stream>>>(h->far.as<double4_32a>(), h->near.as<double4_32a>(),
                                                                  h->idx.as<int>(), h->n, (double *)phi, (double *)grad);
    else
        combine_k<float><<<nblk(h->n, 256), 256, 0, h->stream>>>(h->far.as<double4_32a>(), h->near.as<double4_32a>(),
                                                                 h->idx.as<int>(), h->n, (float *)phi, (float *)grad);
    count_launch(h);
    check_launch("combine");
}

// ---------------------------------------------------------------------------
// FP64 direct sum over all sources for a set of targets; the sources are
// split into nsplit ranges so that a few thousand targets still fill the GPU,
// and the partial sums are added in range order.
// ---------------------------------------------------------------------------
constexpr int DS_T = 128, DS_TILE = 256;

__global__ void __launch_bounds__(DS_T) direct_k(const double *__restrict__ x, const double *__restrict__ q, int64_t n,
                                                 const int64_t *__restrict__ tidx, int64_t nt, int64_t chunk,
                                                 double *__restrict__ part)
{
    __shared__ double4_32a sh[DS_TILE];
    const int64_t t = (int64_t)blockIdx.x * DS_T + threadIdx.x;
    const int split = blockIdx.y;
    const bool act = t < nt;
    const int64_t i = act ? (tidx ? tidx[t] : t) : 0;
    const double xi = act ? x[3 * i] : 0.0, yi = act ? x[3 * i + 1] : 0.0, zi = act ? x[3 * i + 2] : 0.0;
    const int64_t j0 = (int64_t)split * chunk, j1 = min(n, j0 + chunk);
    double p = 0, gx = 0, gy = 0, gz = 0;
    for (int64_t b = j0; b < j1; b += DS_TILE) {
        __syncthreads();
        for (int k = threadIdx.x; k < DS_TILE; k += DS_T) {
            const int64_t j = b + k;
            sh[k] = j < j1 ? make_double4_32a(x[3 * j], x[3 * j + 1], x[3 * j + 2], q[j]) : make_double4_32a(0, 0, 0, 0);
        }
        __syncthreads();
        const int m = (int)min((int64_t)DS_TILE, j1 - b);
        for (int k = 0; k < m; k++) {
            if (b + k == i) continue;
            const double4_32a s = sh[k];
            const double dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            const double r = sqrt(r2);
            const double qr = s.w / r;
            const double qr3 = qr / r2;
            p += qr;
            gx -= qr3 * dx;
            gy -= qr3 * dy;
            gz -= qr3 * dz;
        }
    }
    if (act) {
        double *o = part + ((size_t)split * nt + t) * 4;
        o[0] = p;
        o[1] = gx;
        o[2] = gy;
        o[3] = gz;
    }
}

__global__ void direct_reduce_k(const double *__restrict__ part, int nsplit, int64_t nt, double *__restrict__ phi,
                                double *__restrict__ grad)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double o[4] = {0, 0, 0, 0};
    for (int s = 0; s < nsplit; s++)
        for (int c = 0; c < 4; c++) o[c] += part[((size_t)s * nt + t) * 4 + c];
    phi[t] = o[0];
    if (grad) {
        grad[3 * t] = o[1];
        grad[3 * t + 1] = o[2];
        grad[3 * t + 2] = o[3];
    }
}

void direct_sum(fmm_ctx *h, const double *x, const double *q, int64_t n, const int64_t *tidx, int64_t nt, double *phi,
                double *grad)
{
    cudaStream_t s = h->stream;
    const int64_t tb = (nt + DS_T - 1) / DS_T;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * h->nsm + tb - 1) / tb, (n + 4095) / 4096));
    nsplit = std::min(nsplit, 65535);
    const int64_t chunk = (n + nsplit - 1) / nsplit;
    h->direct_part.ensure(sizeof(double) * 4 * (size_t)nsplit * (size_t)nt);
    dim3 grid((unsigned)tb, (unsigned)nsplit);
    direct_k<<<grid, DS_T, 0, s>>>(x, q, n, tidx, nt, chunk, h->direct_part.as<double>());
    count_launch(h);
    direct_reduce_k<<<nblk(nt, 256), 256, 0, s>>>(h->direct_part.as<double>(), nsplit, nt, phi, grad);
    count_launch(h);
    check_launch("direct");
}

}  // namespace fmm
