// Rotation-based M2L (the paper's GPU code rotates expansions so that the
// translation runs along z, O(p^3) per pair instead of O(p^4); Sec. 2.2 and
// the prior GPU work it cites).
//
// For a translation u = c_L - c_M, a rotation Q takes u to |u| z. In the
// rotated frame the irregular harmonics I_l^mu(|u| z) vanish unless mu = 0,
// where I_l^0 = l! / |u|^(l+1), so the translation couples only equal orders:
//   L'_n^m = (-1)^n sum_{j >= |m|} M'_j^-m (j+n)! / |u|^(j+n+1).
// M' (the multipoles seen from the rotated frame) and L (the locals back in
// the original frame) follow from M and L' by one dense map per degree n,
// (2n+1) x (2n+1) real on the packed coefficients: 2 sum_n (2n+1)^2 + O(p^3)
// multiply-adds per pair.
//
// The maps are built on the host in FP64. On the unit sphere both families
// are multiples of Yt_n^m = P_n^m(cos t) e^{i m f} sqrt((n-m)!/(n+m)!)
// (P without the Condon-Shortley phase): I_n^m = c_nm Yt_n^m and
// R_n^m = Yt_n^m / c_nm with c_nm = sqrt((n+|m|)! (n-|m|)!). A rotation acts
// unitarily on the Yt of one degree. With Q = R_y(-b) R_z(-a) (a, b the
// azimuth and polar angle of u), Yt^m(x) = e^{i m a} sum_m' V_mm'(b) Yt^m'(Qx)
// where V(b) is defined by Yt^m(R_y(b) y) = sum_m' V_mm'(b) Yt^m'(y). With
// this normalisation V_mm'(b) is the Wigner small-d matrix element
// d^n_{m'm}(b); it is evaluated in closed form from its Jacobi-polynomial
// expression (Edmonds, Angular Momentum in Quantum Mechanics, 1957, Eq.
// 4.1.23), once per distinct polar angle, and the azimuth enters as exact
// phases. Then, with U = diag(e^{i m a}) V:
//   M'^m' = sum_m M^m c_m U_mm' / c_m'        (multipoles into the frame)
//   L^m   = sum_m' L'^m' c_m U_mm' / c_m'     (locals back, U^-1 = U^H)

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

using cplx = std::complex<double>;

// offset of degree n's (2n+1) x (2n+1) block in a per-vector map table
int rot_deg_off(int n) { return n * (4 * n * n - 1) / 3; }
int rot_map_size(int p) { return rot_deg_off(p); }

static double fact(int k)
{
    double f = 1;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
}

static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

// Jacobi polynomial P_k^(a,b)(x) by its three-term recurrence in the degree
// (Abramowitz & Stegun 22.7.1), stable for x in [-1, 1]
static double jacobi(int k, int a, int b, double x)
{
    if (k == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((double)(a - b) + (double)(a + b + 2) * x);
    for (int j = 2; j <= k; j++) {
        const double s = (double)(2 * j + a + b);
        const double c1 = 2.0 * j * (double)(j + a + b) * (s - 2.0);
        const double c2 = (s - 1.0) * (double)(a * a - b * b);
        const double c3 = (s - 2.0) * (s - 1.0) * s;
        const double c4 = 2.0 * (double)(j + a - 1) * (double)(j + b - 1) * s;
        const double p2 = ((c2 + c3 * x) * p1 - c4 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// Wigner small-d element d^n_{m'm}(b) from its Jacobi form: with
// k = min(n+m, n-m, n+m', n-m'), the exponents a = |m - m'|,
// c = |m + m'| (= 2n - 2k - a), and the sign (-1)^(m'-m) when m' > m,
//   d = sign sqrt(C(2n-k, k+a) / C(k+c, c)) sin(b/2)^a cos(b/2)^c P_k^(a,c)(cos b)
static double wigner_d(int n, int mp, int m, double b)
{
    const int k = std::min(std::min(n + m, n - m), std::min(n + mp, n - mp));
    int a, lam;
    if (k == n + m || k == n - mp) {
        a = mp - m;
        lam = mp - m;
    } else {
        a = m - mp;
        lam = 0;
    }
    const int c = 2 * n - 2 * k - a;
    const double sgn = (lam & 1) ? -1.0 : 1.0;
    return sgn * std::sqrt(binom(2 * n - k, k + a) / binom(k + c, c)) * std::pow(std::sin(0.5 * b), a) *
           std::pow(std::cos(0.5 * b), c) * jacobi(k, a, c, std::cos(b));
}

// V(b) for every degree n < p: Yt_n^m(R_y(b) y) = sum_m' V_mm' Yt_n^m'(y)
// with V_mm' = d^n_{m'm}(b). V[n] is (2n+1)^2 real, row m + n.
static std::vector<std::vector<double>> vmaps(int p, double b)
{
    std::vector<std::vector<double>> V(p);
    for (int n = 0; n < p; n++) {
        const int K = 2 * n + 1;
        V[n].resize((size_t)K * K);
        for (int m = -n; m <= n; m++)
            for (int mp = -n; mp <= n; mp++) V[n][(size_t)(m + n) * K + (mp + n)] = wigner_d(n, mp, m, b);
    }
    return V;
}

// real packed form of a complex degree-n map given as out^j = sum_i in^i T[i][j]
// (i, j = m + n): column b of the result is the map applied to packed basis vector b
static void packed(int n, const std::vector<cplx> &T, double *out)
{
    const int K = 2 * n + 1;
    std::vector<cplx> in(K), o(K);
    for (int b = 0; b < K; b++) {
        std::fill(in.begin(), in.end(), cplx(0, 0));
        const int m = (b + 1) / 2;
        const cplx e = b == 0 ? cplx(1, 0) : ((b & 1) ? cplx(1, 0) : cplx(0, 1));
        in[n + m] = e;
        if (m) in[n - m] = ((m & 1) ? -1.0 : 1.0) * std::conj(e);
        for (int j = 0; j < K; j++) {
            cplx s(0, 0);
            for (int i = 0; i < K; i++) s += in[i] * T[(size_t)i * K + j];
            o[j] = s;
        }
        out[0 * K + b] = o[n].real();
        for (int mm = 1; mm <= n; mm++) {
            out[(size_t)(2 * mm - 1) * K + b] = o[n + mm].real();
            out[(size_t)(2 * mm) * K + b] = o[n + mm].imag();
        }
    }
}

// V(b) cached per (p, b): the stencil has far fewer polar angles than vectors
static std::mutex g_v_mu;
static std::map<std::pair<int, double>, std::shared_ptr<const std::vector<std::vector<double>>>> g_v_cache;

static std::shared_ptr<const std::vector<std::vector<double>>> vmaps_cached(int p, double b)
{
    const auto key = std::make_pair(p, b);
    {
        std::lock_guard<std::mutex> lk(g_v_mu);
        auto it = g_v_cache.find(key);
        if (it != g_v_cache.end()) return it->second;
    }
    auto v = std::make_shared<const std::vector<std::vector<double>>>(vmaps(p, b));
    std::lock_guard<std::mutex> lk(g_v_mu);
    g_v_cache[key] = v;
    return v;
}

// forward (multipoles into the rotated frame) and backward (locals out of it)
// maps for translation u, each rot_map_size(p) doubles, degree blocks row-major
void rotation_maps(int p, const double u[3], double *A, double *B)
{
    const double rxy = std::hypot(u[0], u[1]);
    const double a = rxy > 0 ? std::atan2(u[1], u[0]) : 0.0, b = std::atan2(rxy, u[2]);
    auto V = vmaps_cached(p, b);
    for (int n = 0; n < p; n++) {
        const int K = 2 * n + 1;
        std::vector<cplx> T((size_t)K * K);
        for (int i = 0; i < K; i++) {
            const int m = i - n;
            const cplx ph = std::polar(1.0, m * a);
            const double cm = std::sqrt(fact(n + std::abs(m)) * fact(n - std::abs(m)));
            for (int j = 0; j < K; j++) {
                const int mp = j - n;
                const double cmp = std::sqrt(fact(n + std::abs(mp)) * fact(n - std::abs(mp)));
                T[(size_t)i * K + j] = cm * ph * (*V)[n][(size_t)i * K + j] / cmp;
            }
        }
        // both directions use T: M'^j = sum_i M^i T_ij, L^i = sum_j L'^j T_ij
        packed(n, T, A + rot_deg_off(n));
        std::vector<cplx> Tt((size_t)K * K);
        for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++) Tt[(size_t)j * K + i] = T[(size_t)i * K + j];
        packed(n, Tt, B + rot_deg_off(n));
    }
}

// the whole rotation M2L on the host, FP64, packed p^2 coefficients
void m2l_rotation_ref(int p, const double u[3], const double *M, double *L)
{
    const int PP = p * p;
    std::vector<double> A(rot_map_size(p)), B(rot_map_size(p)), Mr(PP), Lr(PP);
    rotation_maps(p, u, A.data(), B.data());
    for (int n = 0; n < p; n++) {
        const int K = 2 * n + 1;
        for (int r = 0; r < K; r++) {
            double s = 0;
            for (int c = 0; c < K; c++) s += A[rot_deg_off(n) + (size_t)r * K + c] * M[n * n + c];
            Mr[n * n + r] = s;
        }
    }
    const double d = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    std::vector<double> g(2 * p);
    for (int l = 0; l < 2 * p - 1; l++) g[l] = fact(l) / std::pow(d, l + 1);
    for (int n = 0; n < p; n++)
        for (int m = 0; m <= n; m++) {
            double sr = 0, si = 0;
            for (int j = m; j < p; j++) {
                sr += Mr[re_idx(j, m)] * g[j + n];
                if (m) si += Mr[im_idx(j, m)] * g[j + n];
            }
            const double sg = ((n + m) & 1) ? -1.0 : 1.0;
            Lr[re_idx(n, m)] = sg * sr;
            if (m) Lr[im_idx(n, m)] = -sg * si;
        }
    for (int n = 0; n < p; n++) {
        const int K = 2 * n + 1;
        for (int r = 0; r < K; r++) {
            double s = 0;
            for (int c = 0; c < K; c++) s += B[rot_deg_off(n) + (size_t)r * K + c] * Lr[n * n + c];
            L[n * n + r] = s;
        }
    }
}

}  // namespace fmm

// ---------------------------------------------------------------------------
// device engine
// ---------------------------------------------------------------------------
namespace fmm {

// Device layout of one vector's data (padded so that rows and degree blocks
// start on 16 bytes): A then B, degree n a block of K = 2n+1 rows of
// K4 = K rounded up to 4 entries (zeros past K), then the factors
// g_l = l! / |u|^(l+1), l < 2p - 1, rounded up to 4 entries.
static int k4(int n) { return (2 * n + 1 + 3) & ~3; }
static int rot_blocks(int p)  // entries of A (or B), padded
{
    int s = 0;
    for (int n = 0; n < p; n++) s += (2 * n + 1) * k4(n);
    return s;
}
static int rot_vec_stride(int p) { return 2 * rot_blocks(p) + ((2 * p - 1 + 3) & ~3); }

// one host image per process for each (p, MAC constant, stencil bound)
static std::mutex g_rot_mu;
static std::map<std::tuple<int, double, int>, std::shared_ptr<const std::vector<double>>> g_rot_cache;

static std::shared_ptr<const std::vector<double>> rot_image(fmm_ctx *h)
{
    const auto key = std::make_tuple(h->p, h->cmac, h->st_R);
    {
        std::lock_guard<std::mutex> lk(g_rot_mu);
        auto it = g_rot_cache.find(key);
        if (it != g_rot_cache.end()) return it->second;
    }
    const int p = h->p, RS = rot_map_size(p), nv = h->nV, VS = rot_vec_stride(p), SA = rot_blocks(p);
    std::vector<std::array<int, 3>> vec((size_t)nv);
    const int ne = h->st_off[8];
    for (int e = 0; e < ne; e++) {
        const int *v = &h->st_host[4 * (size_t)e];
        vec[(size_t)(v[3] & 0xffff)] = {v[0], v[1], v[2]};
    }
    auto img = std::make_shared<std::vector<double>>((size_t)nv * VS, 0.0);
    // vectors in parallel on the host cores; u = c_L - c_M = -(source - target)
    const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    // stride t of the vectors: i = t, t + nt, ...
    auto stride = [&](unsigned t) {
        std::vector<double> A(RS), B(RS);
        for (int i = (int)t; i < nv; i += (int)nt) {
            const double u[3] = {-(double)vec[i][0], -(double)vec[i][1], -(double)vec[i][2]};
            rotation_maps(p, u, A.data(), B.data());
            double *o = img->data() + (size_t)i * VS;
            int off = 0;
            for (int n = 0; n < p; n++) {
                const int K = 2 * n + 1, K4 = k4(n);
                for (int r = 0; r < K; r++)
                    for (int c = 0; c < K; c++) {
                        o[off + r * K4 + c] = A[rot_deg_off(n) + r * K + c];
                        o[SA + off + r * K4 + c] = B[rot_deg_off(n) + r * K + c];
                    }
                off += K * K4;
            }
            const double d = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            double g = 1.0 / d;
            for (int l = 0; l < 2 * p - 1; l++) {
                if (l) g *= (double)l / d;
                o[2 * SA + l] = g;
            }
        }
    };
    std::vector<std::thread> pool;
    std::vector<std::exception_ptr> fault(nt);  // an exception stays in its thread until the join
    unsigned started = 0;
    try {
        for (; started < nt; started++)
            pool.emplace_back([&, started] {
                try {
                    stride(started);
                } catch (...) {
                    fault[started] = std::current_exception();
                }
            });
    } catch (...) {
        // a thread could not be created: the strides without a thread run here
    }
    for (unsigned t = started; t < nt; t++) {
        try {
            stride(t);
        } catch (...) {
            fault[t] = std::current_exception();
            break;
        }
    }
    for (auto &th : pool) th.join();
    for (auto &f : fault)
        if (f) std::rethrow_exception(f);
    std::lock_guard<std::mutex> lk(g_rot_mu);
    g_rot_cache[key] = img;
    return img;
}

void rotation_tables_update(fmm_ctx *h, bool fp64)
{
    const int want = fp64 ? 2 : 1;
    if (h->rot_nv == h->nV && h->rot_kind == want && h->rot_tab.p) return;
    auto img = rot_image(h);
    if (fp64) {
        h->rot_tab.ensure(sizeof(double) * img->size());
        FMM_CUDA_TRY(cudaMemcpy(h->rot_tab.p, img->data(), sizeof(double) * img->size(), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(img->size());
        for (size_t i = 0; i < f.size(); i++) f[i] = (float)(*img)[i];
        h->rot_tab.ensure(sizeof(float) * f.size());
        FMM_CUDA_TRY(cudaMemcpy(h->rot_tab.p, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
    }
    h->rot_nv = h->nV;
    h->rot_kind = want;
}

// 16-byte vectors of T and their dot product
template <class T>
struct V16;
template <>
struct V16<float> {
    using type = float4;
    static constexpr int n = 4;
    static __device__ __forceinline__ float dot(float4 a, float4 b, float s)
    {
        return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
    }
};
template <>
struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
    static __device__ __forceinline__ double dot(double2 a, double2 b, double s) { return fma(a.y, b.y, fma(a.x, b.x, s)); }
};

template <class T>
struct RotCfg {
    static constexpr int W = 8;  // warps per CTA, two target cells each
    static constexpr int MINB = sizeof(T) == 4 ? 2 : 1;  // CTAs per SM the registers are sized for
    static constexpr int NK = 8;                       // packed outputs per lane: p^2 <= 256
    static constexpr int NL = 10;                      // padded entries per lane: sum K4 <= 320
};

// One CTA per tile of up to 2W target cells, two per warp. For each stencil
// vector of the tile's set (the prefix that can reach the level), the CTA
// stages the vector's maps and z factors in shared memory; each warp loads
// the M~ of its two cells' sources at that offset (zero where there is none),
// rotates them (lane i: packed output i, 16-byte dot products over its
// degree's padded row, one map entry for both cells), translates along z
// (sums over j of equal order), rotates back and adds into FP64 registers.
// The cells' L~ is written once at the end.
template <class T>
__global__ void __launch_bounds__(32 * RotCfg<T>::W, RotCfg<T>::MINB) m2l_rot_k(int p, const M2LTile *__restrict__ tiles,
                                                             const int *__restrict__ ntiles, const int *__restrict__ tgt,
                                                             const int4 *__restrict__ xyz, const uint64_t *__restrict__ anchor,
                                                             const LevelDesc *__restrict__ ld, const int *__restrict__ map_pool,
                                                             const int4 *__restrict__ st, const int *__restrict__ st_off,
                                                             const T *__restrict__ rot, int VS, int SA, int PP4,
                                                             const T *__restrict__ M, T *__restrict__ L)
{
    using C = RotCfg<T>;
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    if ((int)blockIdx.x >= *ntiles) return;
    const M2LTile td = tiles[blockIdx.x];
    const int PP = p * p;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sTab = reinterpret_cast<T *>(smem_raw);
    const T *sA = sTab, *sB = sTab + SA, *sg = sTab + 2 * SA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *sM[2], *sP[2];
    sM[0] = sTab + VS + (size_t)warp * 4 * PP4;
    sM[1] = sM[0] + PP4;
    sP[0] = sM[0] + 2 * PP4;
    sP[1] = sM[0] + 3 * PP4;
    // the warp's two cells
    int cell[2], rl[2], px[2], py[2], pz[2], ro[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        cell[r] = -1;
        rl[r] = td.level;
        px[r] = py[r] = pz[r] = ro[r] = 0;
        if (2 * warp + r < td.count) {
            cell[r] = tgt[td.start + 2 * warp + r];
            const int4 a = xyz[cell[r]];
            rl[r] = a.w;
            const int sh = FMM_MAXLEVEL - a.w;
            px[r] = a.x >> sh;
            py[r] = a.y >> sh;
            pz[r] = a.z >> sh;
            ro[r] = (px[r] & 1) | ((py[r] & 1) << 1) | ((pz[r] & 1) << 2);
        }
    }
    // this lane's packed outputs i = lane + 32 k: degree n, index a in the
    // degree, position of the entry in the padded layout and of its map rows
    int on[C::NK], oa[C::NK], opos[C::NK], orow[C::NK];
#pragma unroll
    for (int k = 0; k < C::NK; k++) {
        const int i = lane + 32 * k;
        int n = 0, pos = 0, row = 0;
        while ((n + 1) * (n + 1) <= i) {
            const int K4 = (2 * n + 1 + 3) & ~3;
            pos += K4;
            row += (2 * n + 1) * K4;
            n++;
        }
        on[k] = i < PP ? n : -1;
        oa[k] = i - n * n;
        opos[k] = pos + oa[k];
        orow[k] = row + oa[k] * ((2 * n + 1 + 3) & ~3);
    }
    // this lane's padded entries j = lane + 32 t: source index in the packed M~ (-1: padding)
    int lsrc[C::NL];
#pragma unroll
    for (int t = 0; t < C::NL; t++) {
        const int j = lane + 32 * t;
        int n = 0, pos = 0;
        while (n < p && pos + ((2 * n + 1 + 3) & ~3) <= j) {
            pos += (2 * n + 1 + 3) & ~3;
            n++;
        }
        lsrc[t] = (j < PP4 && j - pos < 2 * n + 1) ? n * n + (j - pos) : -1;
    }
    for (int j = lane; j < PP4; j += 32) sP[0][j] = sP[1][j] = T(0);
    double acc[2][C::NK];
#pragma unroll
    for (int k = 0; k < C::NK; k++) acc[0][k] = acc[1][k] = 0.0;

    const int e0 = st_off[td.octant], nvec = st_off[10 + td.octant * (FMM_MAXLEVEL + 1) + td.level];
    for (int e = e0; e < e0 + nvec; e++) {
        const int4 v = st[e];
        __syncthreads();
        {
            const VT *src = reinterpret_cast<const VT *>(rot + (size_t)(v.w & 0xffff) * VS);
            VT *dst = reinterpret_cast<VT *>(sTab);
            for (int i = threadIdx.x; i < VS / VN; i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        int b[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            b[r] = -1;
            if (cell[r] >= 0 && ((v.w >> (16 + ro[r])) & 1))
                b[r] = level_lookup(ld[rl[r]], map_pool, anchor, rl[r], px[r] + v.x, py[r] + v.y, pz[r] + v.z);
        }
        if (b[0] < 0 && b[1] < 0) continue;  // warp-uniform
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int t = 0; t < C::NL; t++) {
                const int j = lane + 32 * t;
                if (j < PP4) sM[r][j] = (b[r] >= 0 && lsrc[t] >= 0) ? M[(size_t)b[r] * PP + lsrc[t]] : T(0);
            }
        __syncwarp();
        // multipoles into the rotated frame
#pragma unroll
        for (int k = 0; k < C::NK; k++) {
            if (on[k] < 0) continue;
            const int n = on[k], K4 = (2 * n + 1 + 3) & ~3, base = opos[k] - oa[k];
            const VT *ar = reinterpret_cast<const VT *>(sA + orow[k]);
            const VT *m0 = reinterpret_cast<const VT *>(sM[0] + base), *m1 = reinterpret_cast<const VT *>(sM[1] + base);
            T s0 = 0, s1 = 0;
            for (int c = 0; c < K4 / VN; c++) {
                const VT w = ar[c];
                s0 = V16<T>::dot(w, m0[c], s0);
                s1 = V16<T>::dot(w, m1[c], s1);
            }
            sP[0][opos[k]] = s0;
            sP[1][opos[k]] = s1;
        }
        __syncwarp();
        // translation along z: only equal orders couple
#pragma unroll
        for (int k = 0; k < C::NK; k++) {
            if (on[k] < 0) continue;
            const int n = on[k], a = oa[k], m = (a + 1) >> 1;
            int pj = 0;
            for (int j = 0; j < m; j++) pj += (2 * j + 1 + 3) & ~3;
            T s0 = 0, s1 = 0;
            for (int j = m; j < p; j++) {
                const T g = sg[j + n];
                s0 += sP[0][pj + a] * g;
                s1 += sP[1][pj + a] * g;
                pj += (2 * j + 1 + 3) & ~3;
            }
            const bool neg = (((n + m) & 1) != 0) != (a > 0 && !(a & 1));
            sM[0][opos[k]] = neg ? -s0 : s0;
            sM[1][opos[k]] = neg ? -s1 : s1;
        }
        __syncwarp();
        // locals back to the original frame
#pragma unroll
        for (int k = 0; k < C::NK; k++) {
            if (on[k] < 0) continue;
            const int n = on[k], K4 = (2 * n + 1 + 3) & ~3, base = opos[k] - oa[k];
            const VT *br = reinterpret_cast<const VT *>(sB + orow[k]);
            const VT *l0 = reinterpret_cast<const VT *>(sM[0] + base), *l1 = reinterpret_cast<const VT *>(sM[1] + base);
            T s0 = 0, s1 = 0;
            for (int c = 0; c < K4 / VN; c++) {
                const VT w = br[c];
                s0 = V16<T>::dot(w, l0[c], s0);
                s1 = V16<T>::dot(w, l1[c], s1);
            }
            acc[0][k] += s0;
            acc[1][k] += s1;
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < 2; r++) {
        if (cell[r] < 0) continue;
#pragma unroll
        for (int k = 0; k < C::NK; k++)
            if (on[k] >= 0) L[(size_t)cell[r] * PP + lane + 32 * k] += (T)acc[r][k];
    }
}

template <class T>
void m2l_rotation(fmm_ctx *h, T *L, const T *M)
{
    using C = RotCfg<T>;
    rotation_tables_update(h, sizeof(T) == 8);
    const int p = h->p, VS = rot_vec_stride(p), SA = rot_blocks(p);
    int PP4 = 0;
    for (int n = 0; n < p; n++) PP4 += k4(n);
    if (PP4 > 32 * C::NL) throw Error{FMM_EINVAL, "rotation M2L: p too large"};
    const size_t smem = sizeof(T) * ((size_t)VS + (size_t)C::W * 4 * PP4);
    ensure_smem((const void *)m2l_rot_k<T>, smem);
    const int *ntiles = reinterpret_cast<const int *>(h->m2l_misc.as<unsigned>() + 24 * (FMM_MAXLEVEL + 1));
    m2l_rot_k<T><<<h->ntiles_max, 32 * C::W, smem, h->work>>>(
        p, h->m2l_tiles.as<M2LTile>(), ntiles, h->m2l_tgt.as<int>(), h->c_xyz.as<int4>(), h->c_anchor.as<uint64_t>(),
        h->lvl_desc.as<LevelDesc>(), h->map_pool.as<int>(), h->st_dev.as<int4>(), stencil_offsets(h),
        h->rot_tab.as<T>(), VS, SA, PP4, M, L);
    count_launch(h);
    check_launch("m2l rotation");
}

template void m2l_rotation<float>(fmm_ctx *, float *, const float *);
template void m2l_rotation<double>(fmm_ctx *, double *, const double *);

bool rotation_m2l_supported(fmm_ctx *h) { return h->p >= 1 && h->p <= 16; }
int rotation_tile_rows(fmm_ctx *h) { return 2 * (h->precision == FMM_FP64 ? RotCfg<double>::W : RotCfg<float>::W); }

}  // namespace fmm
