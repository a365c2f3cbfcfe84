// Apply of the 2D multiscale IBF (Sec. 5.2, eq. f1):
//   u = K_C R_C g + sum over rings, sum over the 12 boxes Q of the ring of
//       U_Q G_Q ... M_Q ... H_Q V_Q^* R_Q g.
// Per ring, every launch covers its 12 boxes.  Lambda of a box is stored in
// i-major pair order (p = i 4^(Lq-l) + j, X box i, Omega box j), element
// ((box m^2 + p) r^2 + t) nc + col.  The 2D transfer from a child grid to
// its parent is the tensor product T_{c1} (x) T_{c2} of the 1D transfer
// matrices, applied as two 1D passes (r^3 instead of r^4 multiply-adds).
#include <algorithm>
#include <cstring>

#include "ibf_2d.h"

namespace ibf {

template <typename Real>
struct C2D;
template <>
struct C2D<float> {
    typedef float2 T;
};
template <>
struct C2D<double> {
    typedef double2 T;
};

template <typename C>
__device__ __forceinline__ C zc()
{
    C r;
    r.x = 0;
    r.y = 0;
    return r;
}
template <typename C>
__device__ __forceinline__ C mulc(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ void addc(C& a, C b)
{
    a.x += b.x;
    a.y += b.y;
}

template <typename Real, int RP>
struct Tmat {
    Real T[2][RP][RP];   // T_c[t][s] = M_t((2c-1)/4 + z_s/2)
};

struct RingArgs {
    double q1[12], q2[12];
    int64_t v_stride, d_stride, m_stride;
    int n, m, Lq, hq, nc;
};

__device__ __forceinline__ int64_t child2(int l, int64_t i, int c)
{
    const int64_t n = 1LL << l;
    return (2 * (i / n) + (c >> 1)) * (2 * n) + 2 * (i % n) + (c & 1);
}

// u[pt + N col] = sum_k KC[pt][k] g[idx(k) + N col]  (the direct centre sum)
template <typename Real>
__global__ void k2_center(const typename C2D<Real>::T* KC, const typename C2D<Real>::T* g,
                          typename C2D<Real>::T* u, int n, int csd, int nc)
{
    typedef typename C2D<Real>::T cx;
    const int64_t N = (int64_t)n * n;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * nc) return;
    const int col = (int)(e % nc);
    const int64_t pt = e / nc;
    const int cc = csd * csd;
    const cx* kr = KC + pt * cc;
    cx acc = zc<cx>();
    for (int k = 0; k < cc; ++k) {
        const int a1 = k / csd + n / 2 - csd / 2, a2 = k % csd + n / 2 - csd / 2;
        addc(acc, mulc(kr[k], g[(int64_t)a1 * n + a2 + N * col]));
    }
    u[pt + N * col] = acc;
}

// Lambda^0[box][j][t][col] = V'[box][j][t] g(q_box + j)
template <typename Real>
__global__ void k2_init(const RingArgs A, int r2, const typename C2D<Real>::T* V, const typename C2D<Real>::T* g,
                        typename C2D<Real>::T* lam)
{
    const int64_t mm = (int64_t)A.m * A.m, N = (int64_t)A.n * A.n;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * mm * r2 * A.nc) return;
    const int col = (int)(e % A.nc);
    const int t = (int)((e / A.nc) % r2);
    const int64_t j = (e / ((int64_t)A.nc * r2)) % mm;
    const int b = (int)(e / ((int64_t)A.nc * r2 * mm));
    const int64_t a1 = (int64_t)(A.q1[b] + 0.5 * A.n) + (j >> A.Lq);
    const int64_t a2 = (int64_t)(A.q2[b] + 0.5 * A.n) + (j & (A.m - 1));
    lam[e] = mulc(V[b * A.v_stride + j * r2 + t], g[a1 * A.n + a2 + N * col]);
}

// One 2D butterfly level l for all 12 boxes.  CTA = (box, unit, rhs tile),
// unit = (X parent ip at level l-1, Omega box j at level Lq-l); inputs
// (ip, child c of j), outputs (child a of ip, j), a, c = 2 c1 + c2.
//   KIND 0 (H): out_a = sum_c (T_{c1} x T_{c2}) (D_{a,c} * in_c)
//   KIND 1 (G): out_a = sum_c D_{a,c} * (T_{a1} x T_{a2})^T in_c
template <typename Real, int RP, int KIND>
__global__ void __launch_bounds__(256) k2_level(const __grid_constant__ Tmat<Real, RP> Tm, const RingArgs A, int l,
                                                const typename C2D<Real>::T* __restrict__ D,
                                                const typename C2D<Real>::T* __restrict__ in,
                                                typename C2D<Real>::T* __restrict__ out, int rt)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP;
    extern __shared__ __align__(16) unsigned char sraw[];
    cx* X = reinterpret_cast<cx*>(sraw);          // [4][R2][rt]
    cx* Wk = X + 4 * R2 * rt;                       // [4][R2][rt]
    cx* Ds = Wk + 4 * R2 * rt;                      // [4][R2]  D_{a,c} for the current a
    const int ntile = (A.nc + rt - 1) / rt;
    const int64_t units = (int64_t)A.m * A.m / 4;
    const int64_t blk = blockIdx.x;
    const int tile = (int)(blk % ntile);
    const int64_t u = (blk / ntile) % units;
    const int b = (int)(blk / (ntile * units));
    const int col0 = tile * rt, ncol = min(rt, A.nc - col0);
    const int64_t nj = 1LL << (2 * (A.Lq - l));          // Omega boxes at level Lq-l
    const int64_t ip = u / nj, j = u % nj;
    const int64_t nC = nj * 4;                            // Omega boxes at level Lq-l+1
    const int64_t mm = (int64_t)A.m * A.m;
    const cx* inb = in + (size_t)b * mm * R2 * A.nc;
    cx* outb = out + (size_t)b * mm * R2 * A.nc;
    const cx* Db = D + (size_t)b * A.d_stride;

    for (int e = threadIdx.x; e < 4 * R2 * rt; e += blockDim.x) {
        const int c = e / (R2 * rt), s = (e / rt) % R2, cl = e % rt;
        const int64_t Cc = child2(A.Lq - l, j, c);
        X[e] = cl < ncol ? inb[((ip * nC + Cc) * R2 + s) * A.nc + col0 + cl] : zc<cx>();
    }
    for (int a = 0; a < 4; ++a) {
        const int64_t Aa = child2(l - 1, ip, a);
        __syncthreads();   // previous a is done with Ds / Wk
        for (int e = threadIdx.x; e < 4 * R2; e += blockDim.x) {
            const int c = e / R2, s = e % R2;
            const int64_t Cc = child2(A.Lq - l, j, c);
            Ds[e] = Db[(Aa * nC + Cc) * R2 + s];
        }
        __syncthreads();
        const int a1 = a >> 1, a2 = a & 1;
        if (KIND == 0) {
            // W[c][s1][t2] = sum_s2 T_{c2}[t2][s2] D_{a,c}[s1,s2] X[c][s1,s2]
            for (int e = threadIdx.x; e < 4 * R2 * rt; e += blockDim.x) {
                const int c = e / (R2 * rt), st = (e / rt) % R2, cl = e % rt;
                const int s1 = st / RP, t2 = st % RP;
                const Real* Tc2 = Tm.T[c & 1][t2];
                cx acc = zc<cx>();
#pragma unroll
                for (int s2 = 0; s2 < RP; ++s2) {
                    const cx y = mulc(Ds[c * R2 + s1 * RP + s2], X[(c * R2 + s1 * RP + s2) * rt + cl]);
                    acc.x += Tc2[s2] * y.x;
                    acc.y += Tc2[s2] * y.y;
                }
                Wk[e] = acc;
            }
            __syncthreads();
            // out_a[t1,t2] = sum_c sum_s1 T_{c1}[t1][s1] W[c][s1][t2]
            for (int e = threadIdx.x; e < R2 * rt; e += blockDim.x) {
                const int t = e / rt, cl = e % rt;
                const int t1 = t / RP, t2 = t % RP;
                cx acc = zc<cx>();
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const Real* Tc1 = Tm.T[c >> 1][t1];
#pragma unroll
                    for (int s1 = 0; s1 < RP; ++s1) {
                        const cx w = Wk[(c * R2 + s1 * RP + t2) * rt + cl];
                        acc.x += Tc1[s1] * w.x;
                        acc.y += Tc1[s1] * w.y;
                    }
                }
                if (cl < ncol) outb[((Aa * nj + j) * R2 + t) * A.nc + col0 + cl] = acc;
            }
        } else {
            // W[c][t1][s2] = sum_s1 T_{a1}[s1][t1] X[c][s1,s2]
            for (int e = threadIdx.x; e < 4 * R2 * rt; e += blockDim.x) {
                const int c = e / (R2 * rt), ts = (e / rt) % R2, cl = e % rt;
                const int t1 = ts / RP, s2 = ts % RP;
                cx acc = zc<cx>();
#pragma unroll
                for (int s1 = 0; s1 < RP; ++s1) {
                    const cx x = X[(c * R2 + s1 * RP + s2) * rt + cl];
                    const Real tv = Tm.T[a1][s1][t1];
                    acc.x += tv * x.x;
                    acc.y += tv * x.y;
                }
                Wk[e] = acc;
            }
            __syncthreads();
            // out_a[t1,t2] = sum_c D_{a,c}[t] sum_s2 T_{a2}[s2][t2] W[c][t1][s2]
            for (int e = threadIdx.x; e < R2 * rt; e += blockDim.x) {
                const int t = e / rt, cl = e % rt;
                const int t1 = t / RP, t2 = t % RP;
                cx acc = zc<cx>();
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    cx z = zc<cx>();
#pragma unroll
                    for (int s2 = 0; s2 < RP; ++s2) {
                        const cx w = Wk[(c * R2 + t1 * RP + s2) * rt + cl];
                        const Real tv = Tm.T[a2][s2][t2];
                        z.x += tv * w.x;
                        z.y += tv * w.y;
                    }
                    addc(acc, mulc(Ds[c * R2 + t], z));
                }
                if (cl < ncol) outb[((Aa * nj + j) * R2 + t) * A.nc + col0 + cl] = acc;
            }
        }
    }
}

// switch at level hq: out[p][t] = sum_s M[p][t][s] in[p][s]
template <typename Real>
__global__ void k2_switch(const RingArgs A, int r2, const typename C2D<Real>::T* M,
                          const typename C2D<Real>::T* in, typename C2D<Real>::T* out)
{
    typedef typename C2D<Real>::T cx;
    const int64_t mm = (int64_t)A.m * A.m;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * mm * r2 * A.nc) return;
    const int col = (int)(e % A.nc);
    const int t = (int)((e / A.nc) % r2);
    const int64_t p = (e / ((int64_t)A.nc * r2)) % mm;
    const int b = (int)(e / ((int64_t)A.nc * r2 * mm));
    const cx* Mr = M + b * A.m_stride + (p * r2 + t) * r2;
    const cx* v = in + ((size_t)(b * mm + p) * r2) * A.nc + col;
    cx acc = zc<cx>();
    for (int s = 0; s < r2; ++s) addc(acc, mulc(Mr[s], v[(int64_t)s * A.nc]));
    out[e] = acc;
}

// u[pt + N col] += sum over the ring's boxes of
//   uph[box][pt] sum_{t1,t2} lw[o1][t1] lw[o2][t2] Lambda^L[box][leaf(pt)][t][col]
template <typename Real, int RP>
__global__ void k2_term(const RingArgs A, const typename C2D<Real>::T* uph, const Real* lw,
                        const typename C2D<Real>::T* lam, typename C2D<Real>::T* u)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP;
    const int64_t N = (int64_t)A.n * A.n, mm = (int64_t)A.m * A.m;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * A.nc) return;
    const int col = (int)(e % A.nc);
    const int64_t pt = e / A.nc;
    const int K = A.n / A.m;
    const int n1 = (int)(pt / A.n), n2 = (int)(pt % A.n);
    const int64_t leaf = (int64_t)(n1 / K) * A.m + n2 / K;
    const Real* w1 = lw + (n1 % K) * RP;
    const Real* w2 = lw + (n2 % K) * RP;
    cx tot = zc<cx>();
    for (int b = 0; b < 12; ++b) {
        const cx* v = lam + ((size_t)(b * mm + leaf) * R2) * A.nc + col;
        cx acc = zc<cx>();
#pragma unroll
        for (int t1 = 0; t1 < RP; ++t1) {
            cx s = zc<cx>();
#pragma unroll
            for (int t2 = 0; t2 < RP; ++t2) {
                const cx x = v[(int64_t)(t1 * RP + t2) * A.nc];
                s.x += w2[t2] * x.x;
                s.y += w2[t2] * x.y;
            }
            acc.x += w1[t1] * s.x;
            acc.y += w1[t1] * s.y;
        }
        addc(tot, mulc(uph[b * N + pt], acc));
    }
    cx o = u[pt + N * col];
    addc(o, tot);
    u[pt + N * col] = o;
}

static inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

template <typename Real, int RP>
static int apply_2d_t(ibf_plan* p, const void* gv, void* uv, int nrhs, cudaStream_t st)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP;
    Plan2D* P = (Plan2D*)p->p2d;
    Tmat<Real, RP> Tm;
    for (int c = 0; c < 2; ++c)
        for (int t = 0; t < RP; ++t)
            for (int s = 0; s < RP; ++s) Tm.T[c][t][s] = (Real)p->T[c][t][s];
    const int64_t N = (int64_t)P->n * P->n;
    static bool attr = false;
    if (!attr) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k2_level<Real, RP, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_level<Real, RP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        attr = true;
    }
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        const int nc = std::min(p->max_nrhs, nrhs - c0);
        const cx* g = (const cx*)gv + N * c0;
        cx* u = (cx*)uv + N * c0;
        prof_start(p, st);
        k2_center<Real><<<nb(N * nc), 256, 0, st>>>((const cx*)P->KC, g, u, P->n, P->center, nc);
        prof_mark(p, st, IBF_K_2D);
        // rhs tile: at most 32 columns and at most ~200 KB of shared memory
        int rt = std::min(32, nc);
        while (rt > 1 && (8 * (size_t)R2 * rt + 4 * R2) * sizeof(cx) > 200 * 1024) rt /= 2;
        const size_t smem = (8 * (size_t)R2 * rt + 4 * R2) * sizeof(cx);
        for (const Ring2D& R : P->rings) {
            RingArgs A;
            memcpy(A.q1, R.q1, sizeof(A.q1));
            memcpy(A.q2, R.q2, sizeof(A.q2));
            A.v_stride = R.v_stride;
            A.d_stride = R.d_stride;
            A.m_stride = R.m_stride;
            A.n = P->n;
            A.m = R.m;
            A.Lq = R.Lq;
            A.hq = R.hq;
            A.nc = nc;
            const int64_t mm = (int64_t)R.m * R.m;
            cx* a = (cx*)P->ws[0];
            cx* b = (cx*)P->ws[1];
            k2_init<Real><<<nb(12 * mm * R2 * nc), 256, 0, st>>>(A, R2, (const cx*)R.V, g, a);
            prof_mark(p, st, IBF_K_2D);
            const int ntile = (nc + rt - 1) / rt;
            const int64_t blocks = 12 * (mm / 4) * ntile;
            for (int l = 1; l <= R.Lq; ++l) {
                if (l <= R.hq)
                    k2_level<Real, RP, 0><<<(unsigned)blocks, 256, smem, st>>>(Tm, A, l, (const cx*)R.D[l], a, b, rt);
                else
                    k2_level<Real, RP, 1><<<(unsigned)blocks, 256, smem, st>>>(Tm, A, l, (const cx*)R.D[l], a, b, rt);
                prof_mark(p, st, IBF_K_2D);
                std::swap(a, b);
                if (l == R.hq) {
                    k2_switch<Real><<<nb(12 * mm * R2 * nc), 256, 0, st>>>(A, R2, (const cx*)R.M, a, b);
                    prof_mark(p, st, IBF_K_2D);
                    std::swap(a, b);
                }
            }
            k2_term<Real, RP><<<nb(N * nc), 256, 0, st>>>(A, (const cx*)R.uph, (const Real*)R.lw, a, u);
            prof_mark(p, st, IBF_K_2D);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "2D apply launch");
}

int apply_2d(ibf_plan* p, const void* g, void* u, int nrhs, cudaStream_t st)
{
    const bool d = p->dtype == IBF_C128;
    switch (p->r) {
    case 5: return d ? apply_2d_t<double, 5>(p, g, u, nrhs, st) : apply_2d_t<float, 5>(p, g, u, nrhs, st);
    case 7: return d ? apply_2d_t<double, 7>(p, g, u, nrhs, st) : apply_2d_t<float, 7>(p, g, u, nrhs, st);
    case 9: return d ? apply_2d_t<double, 9>(p, g, u, nrhs, st) : apply_2d_t<float, 9>(p, g, u, nrhs, st);
    default: return set_error(IBF_ERR_UNSUPPORTED, "2D: r must be 5, 7 or 9");
    }
}

int launches_2d(const ibf_plan* p)
{
    const Plan2D* P = (const Plan2D*)p->p2d;
    int n = 1;
    for (const Ring2D& R : P->rings) n += R.Lq + 3;
    return n;
}

}  // namespace ibf
