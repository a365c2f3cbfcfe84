// Construction of the 2D multiscale IBF (Sec. 5): corona rings of square
// frequency boxes, each with a 2D butterfly of tensor Chebyshev grids, and
// the directly summed centre.  FP64 phases reduced modulo 1 before sincospi;
// compiled with -fmad=false like the 1D construction.
//
// Structured tables per ring (12 boxes each), as in 1D: the left diagonal of
// every H level is merged into the next level's right diagonal, and likewise
// for the G levels, so a level stores one phase per (X box, Omega child box,
// grid point); the switch keeps its full r^2 x r^2 block per pair.
#include <cmath>
#include <cstring>

#include "ibf_2d.h"

namespace ibf {

struct Geo2 {
    int n, r, phase, Lq;
    double m;
    double z[kMaxR];
    // IBF_PHASE_FIO2D_SERIES: frequencies (p_t, q_t) and coefficients of c1, c2
    int nco;
    double pq[kMaxCoef][2], al[2][kMaxCoef], be[2][kMaxCoef];
};

__device__ __forceinline__ double p2(int l) { return (double)(1LL << l); }

// c_d(x) of IBF_PHASE_FIO2D_SERIES: sum_t al cos(2 pi (p x1 + q x2)) + be sin(2 pi (p x1 + q x2))
__device__ __forceinline__ double series2(const Geo2& G, int d, double x1, double x2)
{
    double c = 0.0;
    for (int t = 0; t < G.nco; ++t) {
        const double arg = 2.0 * 3.141592653589793 * (G.pq[t][0] * x1 + G.pq[t][1] * x2);
        c += G.al[d][t] * cos(arg) + G.be[d][t] * sin(arg);
    }
    return c;
}

__device__ __forceinline__ double phi2d(const Geo2& G, double x1, double x2, double k1, double k2)
{
    const double tp = 2.0 * 3.141592653589793;
    const int ph = G.phase;
    if (ph == IBF_PHASE_FIO2D_SERIES) {
        const double a = series2(G, 0, x1, x2) * k1;
        const double b = series2(G, 1, x1, x2) * k2;
        return (x1 * k1 + x2 * k2) + sqrt(a * a + b * b);
    }
    if (ph == IBF_PHASE_FIO2D) {
        double c1 = (2.0 + sin(tp * x1) * sin(tp * x2)) / 16.0;
        double c2 = (2.0 + cos(tp * x1) * cos(tp * x2)) / 16.0;
        double a = c1 * k1;
        double b = c2 * k2;
        return (x1 * k1 + x2 * k2) + sqrt(a * a + b * b);
    }
    if (ph == IBF_PHASE_NUFFT) return x1 * k1 + x2 * k2;
    // IBF_PHASE_SEPARABLE, 2D form
    return 0.75 * sin(tp * x1) * cos(tp * x2) + (0.125 * sqrt(k1 * k1 + k2 * k2) + 0.3 * sin(0.1 * k1 - 0.07 * k2));
}

__device__ __forceinline__ double2 e2(double t)
{
    double th = t - rint(t);
    double s, c;
    sincospi(2.0 * th, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ double lag1(const Geo2& G, int t, double u)
{
    double p = 1.0;
    for (int m = 0; m < G.r; ++m)
        if (m != t) p *= (u - G.z[m]) / (G.z[t] - G.z[m]);
    return p;
}

// X box (l, i): i = i1 2^l + i2, centre ((i1+1/2)/2^l, (i2+1/2)/2^l), side 2^-l
__device__ __forceinline__ void xb(int l, int64_t i, double& c1, double& c2, double& w)
{
    const int64_t n = 1LL << l;
    w = 1.0 / p2(l);
    c1 = ((double)(i / n) + 0.5) * w;
    c2 = ((double)(i % n) + 0.5) * w;
}

// Omega box (l, j) inside the box with lower corner (q1, q2) and side m
__device__ __forceinline__ void wb(const Geo2& G, double q1, double q2, int l, int64_t j, double& c1, double& c2,
                                   double& w)
{
    const int64_t n = 1LL << l;
    w = G.m / p2(l);
    c1 = q1 + ((double)(j / n) + 0.5) * w;
    c2 = q2 + ((double)(j % n) + 0.5) * w;
}

__device__ __forceinline__ int64_t parent2(int l, int64_t i)
{
    const int64_t n = 1LL << l;
    return ((i / n) / 2) * (n / 2) + (i % n) / 2;
}

template <typename C>
__device__ __forceinline__ void put(C* p, double2 v);
template <>
__device__ __forceinline__ void put<double2>(double2* p, double2 v) { *p = v; }
template <>
__device__ __forceinline__ void put<float2>(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

struct Boxes {
    double q1[12], q2[12];
};

// V'[box][j][t] = M^B_t(xi_j) e(Phi(c_root, xi_j)), leaf j holds xi_j = q + (j1, j2)
template <typename C>
__global__ void k2b_V(const Geo2 G, const Boxes Bx, C* V)
{
    const int r2 = G.r * G.r;
    const int64_t mm = (int64_t)G.m * (int64_t)G.m;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * mm * r2) return;
    const int t = (int)(e % r2);
    const int64_t j = (e / r2) % mm;
    const int b = (int)(e / (r2 * mm));
    double cB1, cB2, wB;
    wb(G, Bx.q1[b], Bx.q2[b], G.Lq, j, cB1, cB2, wB);
    const double k1 = Bx.q1[b] + (double)(j >> G.Lq), k2 = Bx.q2[b] + (double)(j & ((1LL << G.Lq) - 1));
    const double w = lag1(G, t / G.r, (k1 - cB1) / wB) * lag1(G, t % G.r, (k2 - cB2) / wB);
    double2 v = e2(phi2d(G, 0.5, 0.5, k1, k2));
    put(V + e, make_double2(w * v.x, w * v.y));
}

// H level l: D[box][i][C][s] = e(Phi(c_{A^l_i}, g^C_s) - Phi(c_{A^{l-1}_{par i}}, g^C_s))
// G level l: D[box][i][C][t] = e(Phi(g^{A^l_i}_t, c_C) - Phi(g^{A^l_i}_t, c_{par C}))
template <typename C>
__global__ void k2b_D(const Geo2 G, const Boxes Bx, int l, int hq, C* D)
{
    const int r2 = G.r * G.r;
    const int64_t ni = 1LL << (2 * l), nC = 1LL << (2 * (G.Lq - l + 1));
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * ni * nC * r2) return;
    const int s = (int)(e % r2);
    const int64_t Cc = (e / r2) % nC;
    const int64_t i = (e / (r2 * nC)) % ni;
    const int b = (int)(e / (r2 * nC * ni));
    const int cl = G.Lq - l + 1;   // Omega level of C
    double d;
    if (l <= hq) {
        double cC1, cC2, wC, cA1, cA2, wA, cP1, cP2, wP;
        wb(G, Bx.q1[b], Bx.q2[b], cl, Cc, cC1, cC2, wC);
        const double g1 = cC1 + wC * G.z[s / G.r], g2 = cC2 + wC * G.z[s % G.r];
        xb(l, i, cA1, cA2, wA);
        xb(l - 1, parent2(l, i), cP1, cP2, wP);
        d = phi2d(G, cA1, cA2, g1, g2) - phi2d(G, cP1, cP2, g1, g2);
    } else {
        double cA1, cA2, wA, cC1, cC2, wC, cR1, cR2, wR;
        xb(l, i, cA1, cA2, wA);
        const double g1 = cA1 + wA * G.z[s / G.r], g2 = cA2 + wA * G.z[s % G.r];
        wb(G, Bx.q1[b], Bx.q2[b], cl, Cc, cC1, cC2, wC);
        wb(G, Bx.q1[b], Bx.q2[b], cl - 1, parent2(cl, Cc), cR1, cR2, wR);
        d = phi2d(G, g1, g2, cC1, cC2) - phi2d(G, g1, g2, cR1, cR2);
    }
    put(D + e, e2(d));
}

// switch at level hq: M[box][p][t][s] = e(Phi(g^A_t, g^B_s) - Phi(c_A, g^B_s) - Phi(g^A_t, c_B))
template <typename C>
__global__ void k2b_M(const Geo2 G, const Boxes Bx, int hq, C* M)
{
    const int r2 = G.r * G.r;
    const int64_t mm = (int64_t)G.m * (int64_t)G.m;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * mm * r2 * r2) return;
    const int s = (int)(e % r2);
    const int t = (int)((e / r2) % r2);
    const int64_t p = (e / ((int64_t)r2 * r2)) % mm;
    const int b = (int)(e / ((int64_t)r2 * r2 * mm));
    const int64_t nj = 1LL << (2 * (G.Lq - hq));
    const int64_t i = p / nj, j = p % nj;
    double cA1, cA2, wA, cB1, cB2, wB;
    xb(hq, i, cA1, cA2, wA);
    wb(G, Bx.q1[b], Bx.q2[b], G.Lq - hq, j, cB1, cB2, wB);
    const double a1 = cA1 + wA * G.z[t / G.r], a2 = cA2 + wA * G.z[t % G.r];
    const double b1 = cB1 + wB * G.z[s / G.r], b2 = cB2 + wB * G.z[s % G.r];
    const double d = phi2d(G, a1, a2, b1, b2) - phi2d(G, cA1, cA2, b1, b2) -
                     phi2d(G, a1, a2, cB1, cB2);
    put(M + e, e2(d));
}

// uph[box][pt] = e(Phi(x_pt, c_Q)) for the grid points x = (n1/n, n2/n)
template <typename C>
__global__ void k2b_U(const Geo2 G, const Boxes Bx, C* U)
{
    const int64_t nx = (int64_t)G.n * G.n;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * nx) return;
    const int64_t pt = e % nx;
    const int b = (int)(e / nx);
    const double x1 = (double)(pt / G.n) / (double)G.n, x2 = (double)(pt % G.n) / (double)G.n;
    const double c1 = Bx.q1[b] + 0.5 * G.m, c2 = Bx.q2[b] + 0.5 * G.m;
    put(U + e, e2(phi2d(G, x1, x2, c1, c2)));
}

// lw[o][t] = M_t((o - K/2)/K): Lagrange weight of a grid point at offset o in
// its leaf of side 1/m (K = n/m points per side)
template <typename R>
__global__ void k2b_lw(const Geo2 G, R* lw)
{
    const int K = G.n / (int)G.m;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * G.r) return;
    const int t = e % G.r, o = e / G.r;
    lw[e] = (R)lag1(G, t, ((double)o - 0.5 * K) / (double)K);
}

// centre kernel KC[pt][k] = e(Phi(x_pt, xi_k)), xi_k = (-c/2 + k1, -c/2 + k2)
template <typename C>
__global__ void k2b_KC(const Geo2 G, int csd, C* KC)
{
    const int64_t nx = (int64_t)G.n * G.n;
    const int64_t cc = (int64_t)csd * csd;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nx * cc) return;
    const int64_t k = e % cc, pt = e / cc;
    const double x1 = (double)(pt / G.n) / (double)G.n, x2 = (double)(pt % G.n) / (double)G.n;
    const double k1 = -0.5 * csd + (double)(k / csd), k2 = -0.5 * csd + (double)(k % csd);
    put(KC + e, e2(phi2d(G, x1, x2, k1, k2)));
}

static inline unsigned nb2(int64_t n) { return (unsigned)((n + 255) / 256); }

static int alloc2(ibf_plan* p, void** ptr, size_t bytes)
{
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_error(IBF_ERR_OOM, "2D plan: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    p->allocations.push_back(*ptr);
    p->factor_bytes += bytes;
    return IBF_OK;
}

template <typename C, typename RE>
static int build_2d_t(ibf_plan* p)
{
    Plan2D* P = (Plan2D*)p->p2d;
    const int n = P->n, r = p->r, r2 = r * r;
    const int64_t nx = (int64_t)n * n;
    int rc;
    Geo2 G;
    memset(&G, 0, sizeof(G));
    G.n = n;
    G.r = r;
    G.phase = p->phase_id;
    for (int t = 0; t < r; ++t) G.z[t] = p->z[t];
    G.nco = (int)p->coef.size() / 6;
    for (int t = 0; t < G.nco; ++t) {
        const double* row = &p->coef[6 * t];
        G.pq[t][0] = row[0];
        G.pq[t][1] = row[1];
        for (int d = 0; d < 2; ++d) {
            G.al[d][t] = row[2 + 2 * d];
            G.be[d][t] = row[3 + 2 * d];
        }
    }
    int64_t nnz = 0;
    // rings: S_t = [-n/2^(t+1), n/2^(t+1))^2 while its side exceeds the centre
    for (int side = n; side > P->center; side /= 2) {
        Ring2D R;
        R.m = side / 4;
        R.Lq = 0;
        while ((1 << R.Lq) < R.m) ++R.Lq;
        R.hq = (R.Lq + 1) / 2;
        const double s0 = -0.5 * side;
        int nb = 0;
        for (int b1 = 0; b1 < 4; ++b1)
            for (int b2 = 0; b2 < 4; ++b2) {
                if (b1 >= 1 && b1 <= 2 && b2 >= 1 && b2 <= 2) continue;
                R.q1[nb] = s0 + b1 * R.m;
                R.q2[nb] = s0 + b2 * R.m;
                ++nb;
            }
        Boxes Bx;
        memcpy(Bx.q1, R.q1, sizeof(Bx.q1));
        memcpy(Bx.q2, R.q2, sizeof(Bx.q2));
        G.m = R.m;
        G.Lq = R.Lq;
        const int64_t mm = (int64_t)R.m * R.m;
        R.v_stride = mm * r2;
        R.d_stride = 4 * mm * r2;
        R.m_stride = mm * (int64_t)r2 * r2;
        if ((rc = alloc2(p, &R.V, sizeof(C) * 12 * R.v_stride))) return rc;
        if ((rc = alloc2(p, &R.M, sizeof(C) * 12 * R.m_stride))) return rc;
        if ((rc = alloc2(p, &R.uph, sizeof(C) * 12 * nx))) return rc;
        if ((rc = alloc2(p, &R.lw, sizeof(RE) * (n / R.m) * r))) return rc;
        R.D.assign(R.Lq + 1, nullptr);
        for (int l = 1; l <= R.Lq; ++l)
            if ((rc = alloc2(p, &R.D[l], sizeof(C) * 12 * R.d_stride))) return rc;
        k2b_V<C><<<nb2(12 * R.v_stride), 256>>>(G, Bx, (C*)R.V);
        for (int l = 1; l <= R.Lq; ++l) k2b_D<C><<<nb2(12 * R.d_stride), 256>>>(G, Bx, l, R.hq, (C*)R.D[l]);
        k2b_M<C><<<nb2(12 * R.m_stride), 256>>>(G, Bx, R.hq, (C*)R.M);
        k2b_U<C><<<nb2(12 * nx), 256>>>(G, Bx, (C*)R.uph);
        k2b_lw<RE><<<nb2((n / R.m) * r), 256>>>(G, (RE*)R.lw);
        nnz += 12 * (R.v_stride + R.Lq * R.d_stride + R.m_stride + nx);
        P->ws_elems = std::max(P->ws_elems, (size_t)12 * mm * r2 * p->max_nrhs);
        P->rings.push_back(R);
    }
    const int64_t cc = (int64_t)P->center * P->center;
    if ((rc = alloc2(p, &P->KC, sizeof(C) * nx * cc))) return rc;
    G.m = 1;
    k2b_KC<C><<<nb2(nx * cc), 256>>>(G, P->center, (C*)P->KC);
    nnz += nx * cc;
    p->nnz = nnz;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "2D construction launch");
    return IBF_OK;
}

int build_2d(ibf_plan* p)
{
    return p->dtype == IBF_C128 ? build_2d_t<double2, double>(p) : build_2d_t<float2, float>(p);
}

}  // namespace ibf
