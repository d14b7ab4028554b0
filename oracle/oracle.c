/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU reference of the 3-D
 * Laplace fast multipole method of Yokota & Barba, "A Tuned and Scalable Fast
 * Multipole Method as a Preeminent Algorithm for Exascale Systems"
 * (arXiv:1106.2176).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check of the package entry
 * file and the CPU-baseline leg of the benchmark may load this library. The
 * GPU library shares no code, header, table or helper with it.
 *
 * What the paper fixes, and where (section of the paper):
 *   - Sec. 2.1: the N-body problem (gravitational / electrostatic, O(N^2)
 *     direct interaction), the hierarchical subdivision of space into near and
 *     far regions, multipole and local expansions of p terms,
 *     and the operator set P2M, M2M, M2L, L2L, L2P plus the direct P2P
 *     near field (Figs. tree5 and flow_chart).
 *   - Sec. 2.2 and Sec. 5: Morton-indexed boxes, sorted particle indices with
 *     start/offset cell ranges, Morton index at a prescribed maximum level.
 *   - Sec. 4: the Laplace kernel.
 * The paper prints no formula. Every definition below is the classical
 * Greengard-Rokhlin spherical-harmonic FMM written out directly; the readings
 * where the paper is silent are listed in the design notes of the repository
 * and restated beside the code that takes them:
 *   - phi_i = sum_{j != i, r_ij > 0} q_j / r_ij ; grad_i = d phi_i / d x_i
 *     (no 1/(4 pi), no softening; coincident pairs are skipped);
 *   - p terms means degrees n = 0 .. p-1;
 *   - R_n^m(x) = r^n P_n^m(cos t) e^{i m f} / (n+m)!,
 *     I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1},
 *     P_n^m without the Condon-Shortley phase, X_n^{-m} = (-1)^m conj(X_n^m);
 *   - root cube from the bounding box, 21-bit quantisation, 63-bit Morton key
 *     with the x bit lowest, stable sort ties broken by input index;
 *   - a cell with more than ncrit particles below level 21 splits into its
 *     non-empty octants; cells numbered breadth first;
 *   - MAC: r_A + r_B < theta * |c_A - c_B| with r the half diagonal, done in
 *     integer half-grid units as 3 (W_A + W_B)^2 < fl(theta^2) * d^2;
 *   - dual tree traversal; on a tie of levels both cells split;
 *   - expansion centres are the geometric box centres.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.
 * No FMA contraction anywhere: quantisation, centres and the MAC must round
 * exactly as written.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_MAXP 40
#define ORC_MAXLEVEL 21

/* ------------------------------------------------------------------------ */
/* factorials                                                                */
/* ------------------------------------------------------------------------ */

#define NFACT (4 * ORC_MAXP + 2)
static double fact_tab[NFACT];
static int fact_ready = 0;

static void init_fact(void)
{
    if (fact_ready) return;
    double f = 1.0;
    fact_tab[0] = 1.0;
    for (int i = 1; i < NFACT; i++) {
        f *= (double)i;
        fact_tab[i] = f;
    }
    fact_ready = 1;
}

static double fact(int k) { return fact_tab[k]; }

/* Index of (n, m), -n <= m <= n, in full storage of P*P complex values. */
static int nm(int n, int m) { return n * n + n + m; }

/* ------------------------------------------------------------------------ */
/* solid harmonics (the expansion basis of Sec. 2.1; classical definitions)  */
/* ------------------------------------------------------------------------ */

static void to_sph(const double x[3], double *r, double *ct, double *st, double *ph)
{
    double rr = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    if (rr == 0.0) {
        *r = 0.0; *ct = 1.0; *st = 0.0; *ph = 0.0;
        return;
    }
    *r = rr;
    *ct = x[2] / rr;
    *st = sqrt(x[0] * x[0] + x[1] * x[1]) / rr;
    *ph = atan2(x[1], x[0]);
}

/* Associated Legendre functions without the Condon-Shortley phase:
 *   P_m^m = (2m-1)!! sin^m,  P_{m+1}^m = (2m+1) cos P_m^m,
 *   (n-m) P_n^m = (2n-1) cos P_{n-1}^m - (n+m-1) P_{n-2}^m.
 * Output row-major Pnm[n*P + m], 0 <= m <= n < P. */
static void legendre(int P, double ct, double st, double *Pnm)
{
    for (int m = 0; m < P; m++) {
        double pmm = 1.0;
        for (int i = 1; i <= m; i++) pmm *= (double)(2 * i - 1) * st;
        Pnm[m * P + m] = pmm;
        if (m + 1 < P) Pnm[(m + 1) * P + m] = (double)(2 * m + 1) * ct * pmm;
        for (int n = m + 2; n < P; n++)
            Pnm[n * P + m] = ((double)(2 * n - 1) * ct * Pnm[(n - 1) * P + m]
                              - (double)(n + m - 1) * Pnm[(n - 2) * P + m]) / (double)(n - m);
    }
}

/* Regular solid harmonics R_n^m(x), n < P, full storage (P*P entries). */
void orc_regular(int P, const double *x, cplx *R)
{
    init_fact();
    double r, ct, st, ph;
    to_sph(x, &r, &ct, &st, &ph);
    double *Pnm = (double *)malloc(sizeof(double) * P * P);
    legendre(P, ct, st, Pnm);
    for (int n = 0; n < P; n++) {
        double rn = pow(r, (double)n);
        for (int m = 0; m <= n; m++) {
            cplx v = rn * Pnm[n * P + m] * cexp(I * (double)m * ph) / fact(n + m);
            R[nm(n, m)] = v;
            R[nm(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
    free(Pnm);
}

/* Irregular solid harmonics I_n^m(x), n < P, full storage; x != 0. */
void orc_irregular(int P, const double *x, cplx *Iout)
{
    init_fact();
    double r, ct, st, ph;
    to_sph(x, &r, &ct, &st, &ph);
    double *Pnm = (double *)malloc(sizeof(double) * P * P);
    legendre(P, ct, st, Pnm);
    for (int n = 0; n < P; n++) {
        double rn1 = pow(r, (double)(n + 1));
        for (int m = 0; m <= n; m++) {
            cplx v = fact(n - m) * Pnm[n * P + m] * cexp(I * (double)m * ph) / rn1;
            Iout[nm(n, m)] = v;
            Iout[nm(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
    free(Pnm);
}

/* ------------------------------------------------------------------------ */
/* direct sum (the quantity the FMM approximates; Sec. 2.1, Sec. 4)          */
/* ------------------------------------------------------------------------ */

/* phi_i = sum_{j != i, r_ij > 0} q_j / r_ij,
 * grad_i = - sum_{j != i, r_ij > 0} q_j (x_i - x_j) / r_ij^3,
 * for the targets tidx[0..nt) (all particles when tidx is NULL), summed over j
 * in index order. x is n*3 row-major. */
void orc_direct(int64_t n, const double *x, const double *q, int64_t nt,
                const int64_t *tidx, double *phi, double *grad)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = tidx ? tidx[t] : t;
        double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = x[3 * i + 0] - x[3 * j + 0];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double qr = q[j] / r;
            double qr3 = qr / r2;
            p += qr;
            gx -= qr3 * dx;
            gy -= qr3 * dy;
            gz -= qr3 * dz;
        }
        phi[t] = p;
        grad[3 * t + 0] = gx;
        grad[3 * t + 1] = gy;
        grad[3 * t + 2] = gz;
    }
}

/* ------------------------------------------------------------------------ */
/* the five translation operators (Sec. 2.1, Fig. flow_chart)               */
/* all expansions in full storage (P*P complex), un-scaled                   */
/* ------------------------------------------------------------------------ */

/* P2M: M_n^m += sum_j q_j conj(R_n^m(x_j - c)). */
void orc_p2m(int P, int64_t n, const double *x, const double *q, const double *c, cplx *M)
{
    cplx *R = (cplx *)malloc(sizeof(cplx) * P * P);
    for (int64_t j = 0; j < n; j++) {
        double d[3] = {x[3 * j] - c[0], x[3 * j + 1] - c[1], x[3 * j + 2] - c[2]};
        orc_regular(P, d, R);
        for (int k = 0; k < P * P; k++) M[k] += q[j] * conj(R[k]);
    }
    free(R);
}

/* M2M, centre c -> c2: M2_n^m += sum_{k<=n, |l|<=k} conj(R_k^l(c - c2)) M_{n-k}^{m-l}. */
void orc_m2m(int P, const cplx *M, const double *c, const double *c2, cplx *M2)
{
    cplx *R = (cplx *)malloc(sizeof(cplx) * P * P);
    double d[3] = {c[0] - c2[0], c[1] - c2[1], c[2] - c2[2]};
    orc_regular(P, d, R);
    for (int n = 0; n < P; n++)
        for (int m = -n; m <= n; m++) {
            cplx s = 0.0;
            for (int k = 0; k <= n; k++)
                for (int l = -k; l <= k; l++) {
                    if (abs(m - l) > n - k) continue;
                    s += conj(R[nm(k, l)]) * M[nm(n - k, m - l)];
                }
            M2[nm(n, m)] += s;
        }
    free(R);
}

/* M2L, multipole at cM -> local at cL, D = cL - cM:
 * L_n^m += (-1)^n sum_{j<P, |k|<=j} M_j^k I_{j+n}^{k+m}(D). */
void orc_m2l(int P, const cplx *M, const double *cM, const double *cL, cplx *L)
{
    int Q = 2 * P - 1;
    cplx *Ih = (cplx *)malloc(sizeof(cplx) * Q * Q);
    double d[3] = {cL[0] - cM[0], cL[1] - cM[1], cL[2] - cM[2]};
    orc_irregular(Q, d, Ih);
    for (int n = 0; n < P; n++)
        for (int m = -n; m <= n; m++) {
            cplx s = 0.0;
            for (int j = 0; j < P; j++)
                for (int k = -j; k <= j; k++)
                    s += M[nm(j, k)] * Ih[nm(j + n, k + m)];
            L[nm(n, m)] += ((n & 1) ? -1.0 : 1.0) * s;
        }
    free(Ih);
}

/* L2L, centre c -> c2, t = c2 - c:
 * L2_k^l += sum_{n>=k, |m|<=n} L_n^m conj(R_{n-k}^{m-l}(t)). */
void orc_l2l(int P, const cplx *L, const double *c, const double *c2, cplx *L2)
{
    cplx *R = (cplx *)malloc(sizeof(cplx) * P * P);
    double t[3] = {c2[0] - c[0], c2[1] - c[1], c2[2] - c[2]};
    orc_regular(P, t, R);
    for (int k = 0; k < P; k++)
        for (int l = -k; l <= k; l++) {
            cplx s = 0.0;
            for (int n = k; n < P; n++)
                for (int m = -n; m <= n; m++) {
                    if (abs(m - l) > n - k) continue;
                    s += L[nm(n, m)] * conj(R[nm(n - k, m - l)]);
                }
            L2[nm(k, l)] += s;
        }
    free(R);
}

/* Value of the full-storage expansion entry X_n^m, zero when |m| > n or n < 0. */
static cplx get(const cplx *X, int n, int m)
{
    if (n < 0 || m > n || m < -n) return 0.0;
    return X[nm(n, m)];
}

/* L2P: phi += Re sum L_n^m conj(R_n^m(x - c)); the gradient from the ladder
 * relations d_z R_n^m = R_{n-1}^m, (d_x - i d_y) conj(R_n^m) = -conj(R_{n-1}^{m+1})
 * i.e. d_x R_n^m = (R_{n-1}^{m-1} - R_{n-1}^{m+1}) / 2,
 *      d_y R_n^m = i (R_{n-1}^{m-1} + R_{n-1}^{m+1}) / 2. */
void orc_l2p(int P, const cplx *L, const double *c, int64_t n, const double *x,
             double *phi, double *grad)
{
    cplx *R = (cplx *)malloc(sizeof(cplx) * P * P);
    for (int64_t j = 0; j < n; j++) {
        double d[3] = {x[3 * j] - c[0], x[3 * j + 1] - c[1], x[3 * j + 2] - c[2]};
        orc_regular(P, d, R);
        cplx p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int a = 0; a < P; a++)
            for (int b = -a; b <= a; b++) {
                cplx Lab = L[nm(a, b)];
                cplx dx = 0.5 * (get(R, a - 1, b - 1) - get(R, a - 1, b + 1));
                cplx dy = 0.5 * I * (get(R, a - 1, b - 1) + get(R, a - 1, b + 1));
                cplx dz = get(R, a - 1, b);
                p += Lab * conj(R[nm(a, b)]);
                gx += Lab * conj(dx);
                gy += Lab * conj(dy);
                gz += Lab * conj(dz);
            }
        phi[j] += creal(p);
        grad[3 * j + 0] += creal(gx);
        grad[3 * j + 1] += creal(gy);
        grad[3 * j + 2] += creal(gz);
    }
    free(R);
}

/* ------------------------------------------------------------------------ */
/* Morton octree (Sec. 2.2: Morton-indexed boxes; Sec. 5: sorted indices     */
/* with start/offset ranges, Morton index at a prescribed maximum level)     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t a, b;
} pair_t;

typedef struct {
    pair_t *v;
    int64_t n, cap;
} pairbuf;

static void pb_push(pairbuf *pb, int64_t a, int64_t b)
{
    if (pb->n == pb->cap) {
        pb->cap = pb->cap ? 2 * pb->cap : 1024;
        pb->v = (pair_t *)realloc(pb->v, sizeof(pair_t) * pb->cap);
    }
    pb->v[pb->n].a = a;
    pb->v[pb->n].b = b;
    pb->n++;
}

static int cmp_pair(const void *pa, const void *pb)
{
    const pair_t *x = (const pair_t *)pa, *y = (const pair_t *)pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx_t;

static int cmp_keyidx(const void *pa, const void *pb)
{
    const keyidx_t *x = (const keyidx_t *)pa, *y = (const keyidx_t *)pb;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

typedef struct {
    int64_t n;
    int ncrit;
    double theta, c; /* c = fl(theta * theta) */
    double origin[3], R0;
    uint32_t *ic;    /* quantised coordinates in input order, n*3 */
    uint64_t *key;   /* sorted keys */
    int64_t *perm;   /* perm[k] = input index of the k-th sorted particle */
    double *xs;      /* sorted positions, n*3 */
    int64_t ncells, cap;
    int32_t *level;
    uint64_t *anchor; /* key of the cell's lowest corner */
    int64_t *acoord;  /* the same corner as integer grid coordinates, 3 per cell */
    int64_t *begin, *end, *child, *parent;
    int32_t *nchild;
    int depth;
    int64_t *p2p_ptr, *p2p_idx, np2p;
    int64_t *m2l_ptr, *m2l_idx, nm2l;
} orc_tree;

/* 63-bit Morton key: bit b of ix -> bit 3b, of iy -> 3b+1, of iz -> 3b+2. */
static uint64_t morton(uint32_t ix, uint32_t iy, uint32_t iz)
{
    uint64_t k = 0;
    for (int b = 0; b < ORC_MAXLEVEL; b++) {
        k |= (uint64_t)((ix >> b) & 1u) << (3 * b);
        k |= (uint64_t)((iy >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((iz >> b) & 1u) << (3 * b + 2);
    }
    return k;
}

static void demorton(uint64_t k, int64_t a[3])
{
    a[0] = a[1] = a[2] = 0;
    for (int b = 0; b < ORC_MAXLEVEL; b++) {
        a[0] |= (int64_t)((k >> (3 * b)) & 1u) << b;
        a[1] |= (int64_t)((k >> (3 * b + 1)) & 1u) << b;
        a[2] |= (int64_t)((k >> (3 * b + 2)) & 1u) << b;
    }
}

static void cell_push(orc_tree *t, int32_t lev, uint64_t anc, int64_t b, int64_t e, int64_t parent)
{
    if (t->ncells == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->level = (int32_t *)realloc(t->level, sizeof(int32_t) * t->cap);
        t->anchor = (uint64_t *)realloc(t->anchor, sizeof(uint64_t) * t->cap);
        t->begin = (int64_t *)realloc(t->begin, sizeof(int64_t) * t->cap);
        t->end = (int64_t *)realloc(t->end, sizeof(int64_t) * t->cap);
        t->child = (int64_t *)realloc(t->child, sizeof(int64_t) * t->cap);
        t->parent = (int64_t *)realloc(t->parent, sizeof(int64_t) * t->cap);
        t->nchild = (int32_t *)realloc(t->nchild, sizeof(int32_t) * t->cap);
        t->acoord = (int64_t *)realloc(t->acoord, sizeof(int64_t) * 3 * t->cap);
    }
    int64_t i = t->ncells++;
    t->level[i] = lev;
    t->anchor[i] = anc;
    t->begin[i] = b;
    t->end[i] = e;
    t->child[i] = -1;
    t->nchild[i] = 0;
    t->parent[i] = parent;
    demorton(anc, t->acoord + 3 * i);
}

/* Multipole acceptance criterion in integer half-grid units:
 * W = 2^(21-l) is the box width in grid units, the centre of a box in
 * half-grid units is 2*anchor + W, the half diagonal is sqrt(3) W, and
 *   accept  <=>  sqrt(3) (W_A + W_B) < theta |D|
 *           <=>  3 (W_A + W_B)^2 < fl(theta^2) * d^2   (one rounding). */
static int mac_accept(const orc_tree *t, int64_t A, int64_t B)
{
    const int64_t *a = t->acoord + 3 * A, *b = t->acoord + 3 * B;
    int64_t WA = (int64_t)1 << (ORC_MAXLEVEL - t->level[A]);
    int64_t WB = (int64_t)1 << (ORC_MAXLEVEL - t->level[B]);
    int64_t d2 = 0;
    for (int k = 0; k < 3; k++) {
        int64_t D = 2 * (a[k] - b[k]) + (WA - WB);
        d2 += D * D;
    }
    double lhs = 3.0 * (double)((WA + WB) * (WA + WB));
    double rhs = t->c * (double)d2;
    return lhs < rhs;
}

/* Dual tree traversal (Sec. 2.1 near/far categorisation). */
static void interact(const orc_tree *t, int64_t A, int64_t B, pairbuf *m2l, pairbuf *p2p)
{
    if (mac_accept(t, A, B)) {
        pb_push(m2l, A, B);
        return;
    }
    int la = t->nchild[A] == 0, lb = t->nchild[B] == 0;
    if (la && lb) {
        pb_push(p2p, A, B);
        return;
    }
    if (!la && (lb || t->level[A] < t->level[B])) {
        for (int64_t a = t->child[A]; a < t->child[A] + t->nchild[A]; a++) interact(t, a, B, m2l, p2p);
        return;
    }
    if (!lb && (la || t->level[B] < t->level[A])) {
        for (int64_t b = t->child[B]; b < t->child[B] + t->nchild[B]; b++) interact(t, A, b, m2l, p2p);
        return;
    }
    for (int64_t a = t->child[A]; a < t->child[A] + t->nchild[A]; a++)
        for (int64_t b = t->child[B]; b < t->child[B] + t->nchild[B]; b++) interact(t, a, b, m2l, p2p);
}

static void to_csr(pairbuf *pb, int64_t ncells, int64_t **ptr, int64_t **idx)
{
    qsort(pb->v, (size_t)pb->n, sizeof(pair_t), cmp_pair);
    *ptr = (int64_t *)calloc((size_t)ncells + 1, sizeof(int64_t));
    *idx = (int64_t *)malloc(sizeof(int64_t) * (pb->n ? pb->n : 1));
    for (int64_t k = 0; k < pb->n; k++) {
        (*ptr)[pb->v[k].a + 1]++;
        (*idx)[k] = pb->v[k].b;
    }
    for (int64_t c = 0; c < ncells; c++) (*ptr)[c + 1] += (*ptr)[c];
}

/* Build the tree and interaction lists for n particles x (n*3, FP64). */
orc_tree *orc_tree_build(int64_t n, const double *x, int ncrit, double theta)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->n = n;
    t->ncrit = ncrit;
    t->theta = theta;
    t->c = theta * theta;

    /* root cube and quantisation */
    double lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = x[k];
        hi[k] = x[k];
    }
    for (int64_t i = 1; i < n; i++)
        for (int k = 0; k < 3; k++) {
            if (x[3 * i + k] < lo[k]) lo[k] = x[3 * i + k];
            if (x[3 * i + k] > hi[k]) hi[k] = x[3 * i + k];
        }
    double R0 = 0.0;
    double cen[3];
    for (int k = 0; k < 3; k++) {
        cen[k] = (lo[k] + hi[k]) * 0.5;
        double h = (hi[k] - lo[k]) * 0.5;
        if (h > R0) R0 = h;
    }
    if (R0 == 0.0) R0 = 1.0;
    for (int k = 0; k < 3; k++) t->origin[k] = cen[k] - R0;
    t->R0 = R0;
    double s = 2097152.0 / (2.0 * R0);
    t->ic = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (n ? n : 1));
    keyidx_t *ki = (keyidx_t *)malloc(sizeof(keyidx_t) * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < 3; k++) {
            double f = floor((x[3 * i + k] - t->origin[k]) * s);
            if (f < 0.0) f = 0.0;
            if (f > 2097151.0) f = 2097151.0;
            t->ic[3 * i + k] = (uint32_t)f;
        }
        ki[i].key = morton(t->ic[3 * i], t->ic[3 * i + 1], t->ic[3 * i + 2]);
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx_t), cmp_keyidx);
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    t->xs = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        t->key[i] = ki[i].key;
        t->perm[i] = ki[i].idx;
        for (int k = 0; k < 3; k++) t->xs[3 * i + k] = x[3 * ki[i].idx + k];
    }
    free(ki);

    /* cells, breadth first: a cell at level l < 21 holding more than ncrit
     * particles splits into its non-empty octants in ascending octant order */
    cell_push(t, 0, 0, 0, n, -1);
    t->depth = 0;
    for (int64_t c = 0; c < t->ncells; c++) {
        int l = t->level[c];
        if (l > t->depth) t->depth = l;
        if (l >= ORC_MAXLEVEL || t->end[c] - t->begin[c] <= ncrit) continue;
        int shift = 3 * (ORC_MAXLEVEL - 1 - l);
        int64_t first = t->ncells;
        int64_t i = t->begin[c];
        for (uint64_t o = 0; o < 8; o++) {
            int64_t b = i;
            while (i < t->end[c] && ((t->key[i] >> shift) & 7u) == o) i++;
            if (i > b) cell_push(t, l + 1, t->anchor[c] | (o << shift), b, i, c);
        }
        t->child[c] = first;
        t->nchild[c] = (int32_t)(t->ncells - first);
    }

    /* interaction lists from the dual traversal, canonical CSR by target */
    pairbuf m2l = {0}, p2p = {0};
    if (n > 0) interact(t, 0, 0, &m2l, &p2p);
    t->nm2l = m2l.n;
    t->np2p = p2p.n;
    to_csr(&m2l, t->ncells, &t->m2l_ptr, &t->m2l_idx);
    to_csr(&p2p, t->ncells, &t->p2p_ptr, &t->p2p_idx);
    free(m2l.v);
    free(p2p.v);
    return t;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    free(t->ic); free(t->key); free(t->perm); free(t->xs);
    free(t->level); free(t->anchor); free(t->begin); free(t->end);
    free(t->child); free(t->parent); free(t->nchild); free(t->acoord);
    free(t->p2p_ptr); free(t->p2p_idx); free(t->m2l_ptr); free(t->m2l_idx);
    free(t);
}

/* sizes[0..6] = ncells, depth, n_p2p_pairs, n_m2l_pairs, n_leaves, n, p2p interactions */
void orc_tree_sizes(const orc_tree *t, int64_t *sizes)
{
    int64_t leaves = 0, inter = 0;
    for (int64_t c = 0; c < t->ncells; c++) {
        if (t->nchild[c] == 0) leaves++;
        for (int64_t k = t->p2p_ptr[c]; k < t->p2p_ptr[c + 1]; k++) {
            int64_t b = t->p2p_idx[k];
            inter += (t->end[c] - t->begin[c]) * (t->end[b] - t->begin[b]);
        }
    }
    sizes[0] = t->ncells;
    sizes[1] = t->depth;
    sizes[2] = t->np2p;
    sizes[3] = t->nm2l;
    sizes[4] = leaves;
    sizes[5] = t->n;
    sizes[6] = inter - t->n; /* self terms excluded */
}

/* box[0..3] = origin x, y, z and R0 */
void orc_tree_box(const orc_tree *t, double *box)
{
    box[0] = t->origin[0];
    box[1] = t->origin[1];
    box[2] = t->origin[2];
    box[3] = t->R0;
}

void orc_tree_particles(const orc_tree *t, uint32_t *ic, uint64_t *key, int64_t *perm)
{
    if (ic) memcpy(ic, t->ic, sizeof(uint32_t) * 3 * t->n);
    if (key) memcpy(key, t->key, sizeof(uint64_t) * t->n);
    if (perm) memcpy(perm, t->perm, sizeof(int64_t) * t->n);
}

void orc_tree_cells(const orc_tree *t, int32_t *level, uint64_t *anchor, int64_t *begin,
                    int64_t *end, int64_t *child, int32_t *nchild, int64_t *parent)
{
    int64_t c = t->ncells;
    if (level) memcpy(level, t->level, sizeof(int32_t) * c);
    if (anchor) memcpy(anchor, t->anchor, sizeof(uint64_t) * c);
    if (begin) memcpy(begin, t->begin, sizeof(int64_t) * c);
    if (end) memcpy(end, t->end, sizeof(int64_t) * c);
    if (child) memcpy(child, t->child, sizeof(int64_t) * c);
    if (nchild) memcpy(nchild, t->nchild, sizeof(int32_t) * c);
    if (parent) memcpy(parent, t->parent, sizeof(int64_t) * c);
}

void orc_tree_lists(const orc_tree *t, int64_t *p2p_ptr, int64_t *p2p_idx, int64_t *m2l_ptr, int64_t *m2l_idx)
{
    int64_t c = t->ncells;
    if (p2p_ptr) memcpy(p2p_ptr, t->p2p_ptr, sizeof(int64_t) * (c + 1));
    if (p2p_idx) memcpy(p2p_idx, t->p2p_idx, sizeof(int64_t) * t->np2p);
    if (m2l_ptr) memcpy(m2l_ptr, t->m2l_ptr, sizeof(int64_t) * (c + 1));
    if (m2l_idx) memcpy(m2l_idx, t->m2l_idx, sizeof(int64_t) * t->nm2l);
}

/* Geometric centre of a cell: origin + (anchor + 2^(20-l)) * (2 R0 / 2^21). */
void orc_cell_centre(const orc_tree *t, int64_t c, double *out)
{
    int64_t a[3];
    demorton(t->anchor[c], a);
    double h = 2.0 * t->R0 / 2097152.0;
    double half = ldexp(1.0, ORC_MAXLEVEL - 1 - t->level[c]);
    for (int k = 0; k < 3; k++) out[k] = t->origin[k] + ((double)a[k] + half) * h;
}

/* ------------------------------------------------------------------------ */
/* FMM evaluation (Fig. flow_chart order: P2M, M2M, M2L, L2L, L2P, P2P)      */
/* ------------------------------------------------------------------------ */

/* Evaluate phi and grad at all particles (input order) for charges q (input
 * order). M and L, when non-NULL, receive the per-cell expansions (ncells*P*P
 * complex, full storage, un-scaled). Returns 0, or -1 on bad arguments. */
int orc_tree_evaluate(const orc_tree *t, const double *q, int P, double *phi, double *grad,
                      cplx *Mout, cplx *Lout)
{
    if (P < 1 || P > ORC_MAXP) return -1;
    init_fact();
    int64_t n = t->n, nc = t->ncells, PP = (int64_t)P * P;
    double *qs = (double *)malloc(sizeof(double) * (n ? n : 1));
    double *ps = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    double *gs = (double *)calloc((size_t)(3 * (n ? n : 1)), sizeof(double));
    cplx *M = (cplx *)calloc((size_t)(nc * PP), sizeof(cplx));
    cplx *L = (cplx *)calloc((size_t)(nc * PP), sizeof(cplx));
    double *cen = (double *)malloc(sizeof(double) * 3 * (nc ? nc : 1));
    for (int64_t i = 0; i < n; i++) qs[i] = q[t->perm[i]];
    for (int64_t c = 0; c < nc; c++) orc_cell_centre(t, c, cen + 3 * c);

    /* P2M at the leaves */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < nc; c++)
        if (t->nchild[c] == 0)
            orc_p2m(P, t->end[c] - t->begin[c], t->xs + 3 * t->begin[c], qs + t->begin[c],
                    cen + 3 * c, M + c * PP);

    /* M2M, deepest level first */
    for (int l = t->depth - 1; l >= 0; l--) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t c = 0; c < nc; c++) {
            if (t->level[c] != l || t->nchild[c] == 0) continue;
            for (int64_t ch = t->child[c]; ch < t->child[c] + t->nchild[c]; ch++)
                orc_m2m(P, M + ch * PP, cen + 3 * ch, cen + 3 * c, M + c * PP);
        }
    }

    /* M2L over every accepted pair */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < nc; c++)
        for (int64_t k = t->m2l_ptr[c]; k < t->m2l_ptr[c + 1]; k++) {
            int64_t b = t->m2l_idx[k];
            orc_m2l(P, M + b * PP, cen + 3 * b, cen + 3 * c, L + c * PP);
        }

    /* L2L, top down: a cell's local expansion includes its parent's */
    for (int l = 0; l < t->depth; l++) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t c = 0; c < nc; c++) {
            if (t->level[c] != l || t->nchild[c] == 0) continue;
            for (int64_t ch = t->child[c]; ch < t->child[c] + t->nchild[c]; ch++)
                orc_l2l(P, L + c * PP, cen + 3 * c, cen + 3 * ch, L + ch * PP);
        }
    }

    /* L2P at the leaves */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < nc; c++)
        if (t->nchild[c] == 0)
            orc_l2p(P, L + c * PP, cen + 3 * c, t->end[c] - t->begin[c], t->xs + 3 * t->begin[c],
                    ps + t->begin[c], gs + 3 * t->begin[c]);

    /* P2P over near leaf pairs; i == j and r == 0 skipped */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < nc; c++)
        for (int64_t k = t->p2p_ptr[c]; k < t->p2p_ptr[c + 1]; k++) {
            int64_t b = t->p2p_idx[k];
            for (int64_t i = t->begin[c]; i < t->end[c]; i++) {
                double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
                for (int64_t j = t->begin[b]; j < t->end[b]; j++) {
                    if (j == i) continue;
                    double dx = t->xs[3 * i] - t->xs[3 * j];
                    double dy = t->xs[3 * i + 1] - t->xs[3 * j + 1];
                    double dz = t->xs[3 * i + 2] - t->xs[3 * j + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2);
                    double qr = qs[j] / r;
                    double qr3 = qr / r2;
                    p += qr;
                    gx -= qr3 * dx;
                    gy -= qr3 * dy;
                    gz -= qr3 * dz;
                }
                ps[i] += p;
                gs[3 * i] += gx;
                gs[3 * i + 1] += gy;
                gs[3 * i + 2] += gz;
            }
        }

    /* back to the input order */
    for (int64_t i = 0; i < n; i++) {
        int64_t o = t->perm[i];
        phi[o] = ps[i];
        for (int k = 0; k < 3; k++) grad[3 * o + k] = gs[3 * i + k];
    }
    if (Mout) memcpy(Mout, M, sizeof(cplx) * nc * PP);
    if (Lout) memcpy(Lout, L, sizeof(cplx) * nc * PP);
    free(qs); free(ps); free(gs); free(M); free(L); free(cen);
    return 0;
}

/* Whole FMM in one call. Returns 0, or -1 on bad arguments. */
int orc_fmm(int64_t n, const double *x, const double *q, int P, double theta, int ncrit,
            double *phi, double *grad)
{
    if (n < 1 || P < 1 || P > ORC_MAXP || !(theta > 0.0 && theta < 1.0) || ncrit < 1) return -1;
    orc_tree *t = orc_tree_build(n, x, ncrit, theta);
    int rc = orc_tree_evaluate(t, q, P, phi, grad, NULL, NULL);
    orc_tree_free(t);
    return rc;
}

int orc_max_p(void) { return ORC_MAXP; }

/* Threads the OpenMP loops over targets use (timing of the CPU baseline on
 * one core and on all cores); results do not depend on it, since each
 * target's sums keep their order. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
