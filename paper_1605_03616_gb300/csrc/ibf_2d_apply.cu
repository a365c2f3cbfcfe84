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
// a b, or conj(a) b when CONJ
template <bool CONJ, typename C>
__device__ __forceinline__ C mulcx(C a, C b)
{
    if (CONJ) a.y = -a.y;
    return mulc(a, b);
}
// acc += a b as a chain of four fused multiply-adds
template <typename C>
__device__ __forceinline__ void cmac(C& acc, C a, C b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <bool CONJ, typename C>
__device__ __forceinline__ void cmacx(C& acc, C a, C b)
{
    if (CONJ) a.y = -a.y;
    cmac(acc, a, b);
}
// Two-lane arithmetic on (re, im) pairs: packed FP32 instructions in single
// precision (one issue slot for both lanes), per-component operations in
// double; a - b is b * (-1) + a rounded once.
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p2fma(float2 w, float2 x, float2 acc) { return __ffma2_rn(w, x, acc); }
__device__ __forceinline__ double2 p2add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 p2sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 p2fma(double2 w, double2 x, double2 acc)
{
    return make_double2(fma(w.x, x.x, acc.x), fma(w.y, x.y, acc.y));
}

struct RingArgs {
    double q1[12], q2[12];
    int64_t v_stride, d_stride, m_stride;
    int n, m, Lq, hq, nc;
};

// u[pt + N col] = sum_k KC[pt][k] g[idx(k) + N col]  (the direct centre sum)
// CTA = (128 points, rhs tile): the centre entries of g for the tile are
// staged once, KC rows stream through shared memory in chunks of 32; thread
// (point, column parity) keeps rt/2 outputs so stores run along the points.
template <typename Real>
__global__ void __launch_bounds__(256) k2_center(const typename C2D<Real>::T* __restrict__ KC,
                                                 const typename C2D<Real>::T* __restrict__ g,
                                                 typename C2D<Real>::T* __restrict__ u, int n, int csd, int nc, int rt)
{
    typedef typename C2D<Real>::T cx;
    constexpr int PT = 128, KCH = 32, CPT = 16;
    extern __shared__ __align__(16) unsigned char sraw[];
    const int cc = csd * csd;
    cx* Gs = reinterpret_cast<cx*>(sraw);   // [cc][rt]
    cx* Ks = Gs + (size_t)cc * rt;            // [PT][KCH + 1]
    const int64_t N = (int64_t)n * n;
    const int ntile = (nc + rt - 1) / rt;
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t pt0 = (blockIdx.x / ntile) * PT;
    const int col0 = tile * rt, ncol = min(rt, nc - col0);
    for (int e = threadIdx.x; e < cc * rt; e += blockDim.x) {
        const int cl = e / cc, k = e % cc;
        const int a1 = k / csd + n / 2 - csd / 2, a2 = k % csd + n / 2 - csd / 2;
        Gs[k * rt + cl] = cl < ncol ? g[(int64_t)a1 * n + a2 + N * (col0 + cl)] : zc<cx>();
    }
    const int pl = threadIdx.x % PT, cg = threadIdx.x / PT;
    cx acc[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) acc[k] = zc<cx>();
    for (int kc = 0; kc < cc; kc += KCH) {
        __syncthreads();
        for (int e = threadIdx.x; e < PT * KCH; e += blockDim.x) {
            const int pr = e / KCH, kk = e % KCH;
            Ks[pr * (KCH + 1) + kk] = kc + kk < cc ? KC[(pt0 + pr) * cc + kc + kk] : zc<cx>();
        }
        __syncthreads();
        const int kend = min(KCH, cc - kc);
        for (int kk = 0; kk < kend; ++kk) {
            const cx kv = Ks[pl * (KCH + 1) + kk];
            const cx* gr = Gs + (kc + kk) * rt + cg;
#pragma unroll
            for (int k = 0; k < CPT; ++k)
                if (cg + 2 * k < rt) cmac(acc[k], kv, gr[2 * k]);
        }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = cg + 2 * k;
        if (c < ncol) u[pt0 + pl + N * (col0 + c)] = acc[k];
    }
}

// One 2D butterfly level l for all 12 boxes.  CTA = (box, unit, rhs tile),
// unit = (X parent ip at level l-1, Omega box j at level Lq-l); inputs
// (ip, child c of j), outputs (child a of ip, j), a, c = 2 c1 + c2.
//   H: out_a = sum_c (T_{c1} x T_{c2}) (D_{a,c} * in_c)
//   G: out_a = sum_c D_{a,c} * (T_{a1} x T_{a2})^T in_c

// Even/odd weights of T_0 (T_1 = J T_0 J, as in 1D): H form rows by input
// index (PmT[s][t], QmT[s][t]), G form rows by output index (E[t][s], F[t][s]).
// Each weight is stored as a (w, w) pair, so one two-lane multiply-add
// applies it to a complex value.
template <typename Real, int RP>
struct EO2 {
    static constexpr int HR = (RP + 1) / 2, HQ = RP / 2;
    typedef typename C2D<Real>::T P;
    P PmT[RP][HR];
    P QmT[RP][HQ];
    P E[RP][HR];
    P F[RP][HQ];
};

// Child of box i at quadtree level l (side 2^l boxes per axis), c = 2 c1 + c2.
__device__ __forceinline__ int64_t child2s(int l, int64_t i, int c)
{
    return ((2 * (i >> l) + (c >> 1)) << (l + 1)) + 2 * (i & ((1LL << l) - 1)) + (c & 1);
}

// Asynchronous 8- or 16-byte global -> shared copy; !valid writes zeros.
__device__ __forceinline__ void cp_async_cx(float2* dst, const float2* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_cx(double2* dst, const double2* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

// Shared prologue of both level kernels: the CTA's unit and rhs tile, its
// four input blocks X[ki][s][col] and all sixteen diagonals, staged as
// Ds[ko][ki][s] for kernel output ko and kernel input ki.  Forward
// (ADJ = false) the inputs are the unit's four pairs (ip, child c of j) of
// level l-1 and the outputs its four pairs (child a of ip, j) of level l,
// Ds[a][c] = D_{a,c}.  The adjoint runs the other way: inputs the level-l
// pairs (child a of ip, j), outputs the level-(l-1) pairs (ip, child c of j),
// Ds[c][a] = D_{a,c}, conjugated by the kernels when they use it.
template <typename Real, int RP, bool ADJ = false>
struct LevelTile {
    typedef typename C2D<Real>::T cx;
    static constexpr int R2 = RP * RP;
    int64_t ip, j, nj;
    int col0, ncol, Lq, l;
    cx* outb;
    // pair index of kernel output ko (the block start is its R2 nc elements)
    __device__ int64_t out_pair(int ko) const
    {
        return ADJ ? ip * nj * 4 + child2s(Lq - l, j, ko) : child2s(l - 1, ip, ko) * nj + j;
    }
    // With g0 != nullptr (level 1) the inputs are Lambda^0 = V' g formed here
    // from the box's V table and g, instead of read from the workspace.
    __device__ void stage(const RingArgs& A, int l, const cx* D, const cx* in, cx* out, int rt, int lrt, cx* X,
                          cx* Ds, const cx* g0 = nullptr, const cx* V0 = nullptr)
    {
        const int ntile = (A.nc + rt - 1) >> lrt;
        const int64_t units = (int64_t)A.m * A.m / 4;
        const int tile = (int)(blockIdx.x % ntile);
        const int64_t u = (blockIdx.x / ntile) % units;
        const int b = (int)(blockIdx.x / (ntile * units));
        col0 = tile << lrt;
        ncol = min(rt, A.nc - col0);
        Lq = A.Lq;
        this->l = l;
        const int ql = 2 * (A.Lq - l);
        nj = 1LL << ql;
        ip = u >> ql;
        j = u & (nj - 1);
        const int64_t nC = nj * 4, mm = (int64_t)A.m * A.m;
        const cx* inb = in + (size_t)b * mm * R2 * A.nc + col0;
        outb = out + (size_t)b * mm * R2 * A.nc + col0;
        const cx* Db = D + (size_t)b * A.d_stride;
        const int cl = threadIdx.x & (rt - 1), srow = threadIdx.x >> lrt, sstep = blockDim.x >> lrt;
        // asynchronous copies: every load of the tile is in flight at once;
        // columns past the tile's end are zero-filled (source size 0)
        cx* Vs = Ds + 16 * R2;   // level 1 only: [4 c][R2] V rows, [4 c][rt] g values
        cx* Gs = Vs + 4 * R2;
        if (g0) {
            const int64_t N = (int64_t)A.n * A.n;
            const int64_t o1 = (int64_t)(A.q1[b] + 0.5 * A.n), o2 = (int64_t)(A.q2[b] + 0.5 * A.n);
            for (int e = threadIdx.x; e < 4 * R2; e += blockDim.x) {
                const int c = e / R2, sidx = e - c * R2;
                cp_async_cx(Vs + e, V0 + b * A.v_stride + child2s(A.Lq - 1, j, c) * R2 + sidx, true);
            }
            for (int e = threadIdx.x; e < 4 * rt; e += blockDim.x) {
                const int c = e >> lrt, k = e & (rt - 1);
                const int64_t leaf = child2s(A.Lq - 1, j, c);
                const cx* gp = g0 + (o1 + (leaf >> A.Lq)) * A.n + o2 + (leaf & (A.m - 1)) + N * col0;
                cp_async_cx(Gs + e, k < ncol ? gp + N * k : gp, k < ncol);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t pin = ADJ ? child2s(l - 1, ip, c) * nj + j : ip * nC + child2s(A.Lq - l, j, c);
                const cx* src = inb + pin * R2 * A.nc;
                for (int sidx = srow; sidx < R2; sidx += sstep)
                    cp_async_cx(X + (c * R2 + sidx) * rt + cl, cl < ncol ? src + (int64_t)sidx * A.nc + cl : src,
                                cl < ncol);
            }
        }
        for (int e = threadIdx.x; e < 16 * R2; e += blockDim.x) {
            const int ac = e / R2, sidx = e - ac * R2;
            const int a = ADJ ? (ac & 3) : (ac >> 2), c = ADJ ? (ac >> 2) : (ac & 3);
            cp_async_cx(Ds + e, Db + (child2s(l - 1, ip, a) * nC + child2s(A.Lq - l, j, c)) * R2 + sidx, true);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        if (g0) {
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 4; ++c)
                for (int sidx = srow; sidx < R2; sidx += sstep)
                    X[(c * R2 + sidx) * rt + cl] = mulc(Vs[c * R2 + sidx], Gs[c * rt + cl]);
        }
    }
};

// Level kernels: 2 r rt threads with rt = 16 (FP32) or 8 (FP64) columns.
template <typename Real, int RP>
constexpr int k2_level_threads() { return (2 * RP * (sizeof(Real) == 8 ? 8 : 16) + 31) / 32 * 32; }
template <typename Real, int RP>
constexpr int k2_level_blocks() { return sizeof(Real) == 8 ? 1 : (RP > 7 ? 2 : 3); }

// 2D H level, even/odd in both tensor directions.  For output a:
//   W_{c1}[s1][.] = P T_0 (Y_{c1,0}[s1] + J Y_{c1,1}[s1]) + Q T_0 (Y_{c1,0}[s1] - J Y_{c1,1}[s1]),
//   Y_c = D_{a,c} * X_c, then the same over s1 for c1 = 0, 1.  Two outputs
// per pass: 4 r rt tasks in pass 1, 2 r rt in pass 2, 2 r rt threads.
template <typename Real, int RP, bool ADJ>
__global__ void __launch_bounds__(k2_level_threads<Real, RP>(), k2_level_blocks<Real, RP>())
    k2_level_h(const __grid_constant__ EO2<Real, RP> W, const RingArgs A, int l,
               const typename C2D<Real>::T* __restrict__ D, const typename C2D<Real>::T* __restrict__ in,
               typename C2D<Real>::T* __restrict__ out, int rt, int lrt, const typename C2D<Real>::T* __restrict__ g0,
               const typename C2D<Real>::T* __restrict__ V0)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP, HR = EO2<Real, RP>::HR, HQ = EO2<Real, RP>::HQ;
    extern __shared__ __align__(16) unsigned char sraw[];
    cx* X = reinterpret_cast<cx*>(sraw);            // [4 c][R2][rt]
    cx* Ws = X + 4 * R2 * rt;                         // [2 a][2 c1][RP s1][RP t2][rt]
    cx* Ds = Ws + 4 * R2 * rt;                        // [4 a][4 c][R2] (+ level-1 V rows and g)
    LevelTile<Real, RP, ADJ> T;
    T.stage(A, l, D, in, out, rt, lrt, X, Ds, g0, V0);
    const int msk = rt - 1;
    for (int a0 = 0; a0 < 4; a0 += 2) {
        __syncthreads();
        // pass 1: task (ah, c1, s1, col) -> W_{a0+ah, c1}[s1][t2], t2 = 0..RP-1
        for (int e = threadIdx.x; e < 4 * RP * rt; e += blockDim.x) {
            const int cl = e & msk, q = e >> lrt;
            const int s1 = q % RP, r4 = q / RP, c1 = r4 & 1, ah = r4 >> 1;
            const int c0 = 2 * c1, cc1 = 2 * c1 + 1;   // children (c1, 0) and (c1, 1)
            const cx* d0 = Ds + ((a0 + ah) * 4 + c0) * R2 + s1 * RP;
            const cx* d1 = Ds + ((a0 + ah) * 4 + cc1) * R2 + s1 * RP;
            const cx* x0 = X + (c0 * R2 + s1 * RP) * rt + cl;
            const cx* x1 = X + (cc1 * R2 + s1 * RP) * rt + cl;
            cx we[HR], wo[HQ > 0 ? HQ : 1];
#pragma unroll
            for (int t = 0; t < HR; ++t) we[t] = zc<cx>();
#pragma unroll
            for (int t = 0; t < HQ; ++t) wo[t] = zc<cx>();
#pragma unroll
            for (int s2 = 0; s2 < RP; ++s2) {
                const cx y0 = mulcx<ADJ>(d0[s2], x0[s2 * rt]);
                const cx y1 = mulcx<ADJ>(d1[RP - 1 - s2], x1[(RP - 1 - s2) * rt]);
                const cx pv = p2add(y0, y1), mv = p2sub(y0, y1);
#pragma unroll
                for (int t = 0; t < HR; ++t) we[t] = p2fma(W.PmT[s2][t], pv, we[t]);
#pragma unroll
                for (int t = 0; t < HQ; ++t) wo[t] = p2fma(W.QmT[s2][t], mv, wo[t]);
            }
            cx* wd = Ws + (((ah * 2 + c1) * RP + s1) * RP) * rt + cl;
#pragma unroll
            for (int t = 0; t < HQ; ++t) {
                wd[t * rt] = p2add(we[t], wo[t]);
                wd[(RP - 1 - t) * rt] = p2sub(we[t], wo[t]);
            }
            if (RP & 1) wd[HQ * rt] = we[HQ];
        }
        __syncthreads();
        // pass 2: task (ah, t2, col) -> out_{a0+ah}[t1][t2], t1 = 0..RP-1
        for (int e = threadIdx.x; e < 2 * RP * rt; e += blockDim.x) {
            const int cl = e & msk, q = e >> lrt;
            const int t2 = q % RP, ah = q / RP;
            const cx* w0 = Ws + ((ah * 2 + 0) * R2 + t2) * rt + cl;
            const cx* w1 = Ws + ((ah * 2 + 1) * R2 + t2) * rt + cl;
            cx we[HR], wo[HQ > 0 ? HQ : 1];
#pragma unroll
            for (int t = 0; t < HR; ++t) we[t] = zc<cx>();
#pragma unroll
            for (int t = 0; t < HQ; ++t) wo[t] = zc<cx>();
#pragma unroll
            for (int s1 = 0; s1 < RP; ++s1) {
                const cx v0 = w0[s1 * RP * rt];
                const cx v1 = w1[(RP - 1 - s1) * RP * rt];
                const cx pv = p2add(v0, v1), mv = p2sub(v0, v1);
#pragma unroll
                for (int t = 0; t < HR; ++t) we[t] = p2fma(W.PmT[s1][t], pv, we[t]);
#pragma unroll
                for (int t = 0; t < HQ; ++t) wo[t] = p2fma(W.QmT[s1][t], mv, wo[t]);
            }
            if (cl < T.ncol) {
                cx* od = T.outb + (T.out_pair(a0 + ah) * R2 + t2) * A.nc + cl;
#pragma unroll
                for (int t = 0; t < HQ; ++t) {
                    od[(int64_t)(t * RP) * A.nc] = p2add(we[t], wo[t]);
                    od[(int64_t)((RP - 1 - t) * RP) * A.nc] = p2sub(we[t], wo[t]);
                }
                if (RP & 1) od[(int64_t)(HQ * RP) * A.nc] = we[HQ];
            }
        }
    }
}

// 2D G level: both tensor directions use e/f (T_0^T x = e + f,
// T_1^T x = J(e - f)) so the four outputs share one pass per input.  Two
// inputs per pass 1 (2 r rt tasks); thread (a1, t1, col) keeps
// out_{(a1,a2)}[t1][.] for a2 = 0, 1 in registers over all four inputs.
template <typename Real, int RP, bool ADJ>
__global__ void __launch_bounds__(k2_level_threads<Real, RP>(), k2_level_blocks<Real, RP>())
    k2_level_g(const __grid_constant__ EO2<Real, RP> W, const RingArgs A, int l,
               const typename C2D<Real>::T* __restrict__ D, const typename C2D<Real>::T* __restrict__ in,
               typename C2D<Real>::T* __restrict__ out, int rt, int lrt)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP, HR = EO2<Real, RP>::HR, HQ = EO2<Real, RP>::HQ;
    extern __shared__ __align__(16) unsigned char sraw[];
    cx* X = reinterpret_cast<cx*>(sraw);            // [4 c][R2][rt]
    cx* Zs = X + 4 * R2 * rt;                         // [2 ch][2 a1][RP t1][RP s2][rt]
    cx* Ds = Zs + 4 * R2 * rt;                        // [4 a][4 c][R2]
    LevelTile<Real, RP, ADJ> T;
    T.stage(A, l, D, in, out, rt, lrt, X, Ds);
    const int msk = rt - 1;
    const bool mine = threadIdx.x < 2 * RP * rt;
    const int mcl = threadIdx.x & msk, mq = threadIdx.x >> lrt;
    const int mt1 = mq % RP, ma1 = mq / RP;
    cx acc[2][RP];
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
        for (int t = 0; t < RP; ++t) acc[a2][t] = zc<cx>();
    for (int c0 = 0; c0 < 4; c0 += 2) {
        __syncthreads();
        // pass 1: task (ch, s2, col): Z_{ch, a1}[t1][s2] for a1 = 0, 1 from column s2 of X_{c0+ch}
        for (int e = threadIdx.x; e < 2 * RP * rt; e += blockDim.x) {
            const int cl = e & msk, q = e >> lrt;
            const int s2 = q % RP, ch = q / RP;
            const cx* xc = X + ((c0 + ch) * R2 + s2) * rt + cl;
            cx xe[HR], xo[HQ > 0 ? HQ : 1];
#pragma unroll
            for (int s1 = 0; s1 < HQ; ++s1) {
                const cx lo = xc[s1 * RP * rt], hi = xc[(RP - 1 - s1) * RP * rt];
                xe[s1] = p2add(lo, hi);
                xo[s1] = p2sub(lo, hi);
            }
            if (RP & 1) xe[HQ] = xc[HQ * RP * rt];
            cx* z = Zs + (ch * 2 * R2 + s2) * rt + cl;
#pragma unroll
            for (int t1 = 0; t1 < RP; ++t1) {
                cx ev = zc<cx>(), fv = zc<cx>();
#pragma unroll
                for (int sidx = 0; sidx < HR; ++sidx) ev = p2fma(W.E[t1][sidx], xe[sidx], ev);
#pragma unroll
                for (int sidx = 0; sidx < HQ; ++sidx) fv = p2fma(W.F[t1][sidx], xo[sidx], fv);
                z[(t1 * RP) * rt] = p2add(ev, fv);
                z[(R2 + (RP - 1 - t1) * RP) * rt] = p2sub(ev, fv);
            }
        }
        __syncthreads();
        // pass 2: task (a1, t1, col), both inputs of this pass
        if (mine) {
#pragma unroll 1
            for (int ch = 0; ch < 2; ++ch) {
                const int c = c0 + ch;
                const cx* zr = Zs + ((ch * 2 + ma1) * R2 + mt1 * RP) * rt + mcl;
                cx xe[HR], xo[HQ > 0 ? HQ : 1];
#pragma unroll
                for (int s2 = 0; s2 < HQ; ++s2) {
                    const cx lo = zr[s2 * rt], hi = zr[(RP - 1 - s2) * rt];
                    xe[s2] = p2add(lo, hi);
                    xo[s2] = p2sub(lo, hi);
                }
                if (RP & 1) xe[HQ] = zr[HQ * rt];
                const cx* d0 = Ds + ((2 * ma1 + 0) * 4 + c) * R2 + mt1 * RP;
                const cx* d1 = Ds + ((2 * ma1 + 1) * 4 + c) * R2 + mt1 * RP;
#pragma unroll
                for (int t2 = 0; t2 < RP; ++t2) {
                    cx ev = zc<cx>(), fv = zc<cx>();
#pragma unroll
                    for (int sidx = 0; sidx < HR; ++sidx) ev = p2fma(W.E[t2][sidx], xe[sidx], ev);
#pragma unroll
                    for (int sidx = 0; sidx < HQ; ++sidx) fv = p2fma(W.F[t2][sidx], xo[sidx], fv);
                    cmacx<ADJ>(acc[0][t2], d0[t2], p2add(ev, fv));
                    cmacx<ADJ>(acc[1][RP - 1 - t2], d1[RP - 1 - t2], p2sub(ev, fv));
                }
            }
        }
    }
    if (mine && mcl < T.ncol) {
#pragma unroll
        for (int a2 = 0; a2 < 2; ++a2) {
            cx* od = T.outb + (T.out_pair(2 * ma1 + a2) * R2 + mt1 * RP) * A.nc + mcl;
#pragma unroll
            for (int t2 = 0; t2 < RP; ++t2) od[(int64_t)t2 * A.nc] = acc[a2][t2];
        }
    }
}

// Switch at level hq: out[p][t] = sum_s M[p][t][s] in[p][s].  CTA = (box,
// pair p, 32-column tile): M[p] (r^2 x r^2) and the pair's input tile are
// staged by asynchronous copies; thread (column group cg, row group tg)
// keeps outputs t = tg + 16k for the columns cg + 8q (q < 4) in registers,
// so one shared load of M serves four columns and one of x four rows.
template <typename Real, int RP, bool ADJ = false>
__global__ void __launch_bounds__(128) k2_switch(const RingArgs A, const typename C2D<Real>::T* __restrict__ M,
                                                 const typename C2D<Real>::T* __restrict__ in,
                                                 typename C2D<Real>::T* __restrict__ out)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP, CW = 32, TG = 16, KT = (R2 + TG - 1) / TG;
    extern __shared__ __align__(16) unsigned char sraw[];
    cx* Ms = reinterpret_cast<cx*>(sraw);   // [R2][R2]
    cx* Xs = Ms + R2 * R2;                    // [R2][CW]
    const int ntile = (A.nc + CW - 1) / CW;
    const int64_t mm = (int64_t)A.m * A.m;
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t bp = blockIdx.x / ntile;    // b * mm + p
    const int b = (int)(bp / mm);
    const int64_t p = bp % mm;
    const int col0 = tile * CW, ncol = min(CW, A.nc - col0);
    const cx* Mr = M + b * A.m_stride + p * R2 * R2;
    if (!ADJ) {
        for (int e = threadIdx.x; e < R2 * R2; e += blockDim.x) cp_async_cx(Ms + e, Mr + e, true);
    } else {
        // adjoint: out[s] = sum_t conj(M[t][s]) in[t], staged as the conjugate transpose
        for (int e = threadIdx.x; e < R2 * R2; e += blockDim.x) {
            const int t = e / R2, sidx = e - t * R2;
            cx v = Mr[e];
            v.y = -v.y;
            Ms[sidx * R2 + t] = v;
        }
    }
    const cx* xin = in + (size_t)bp * R2 * A.nc + col0;
    for (int e = threadIdx.x; e < R2 * CW; e += blockDim.x) {
        const int sidx = e >> 5, cl = e & 31;
        cp_async_cx(Xs + e, cl < ncol ? xin + (int64_t)sidx * A.nc + cl : xin, cl < ncol);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int cg = threadIdx.x & 7, tg = threadIdx.x >> 3;
    cx acc[KT][4];
#pragma unroll
    for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[k][q] = zc<cx>();
#pragma unroll 7
    for (int sidx = 0; sidx < R2; ++sidx) {
        cx x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = Xs[sidx * CW + cg + 8 * q];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int t = tg + k * TG;
            if (t < R2) {
                const cx m = Ms[t * R2 + sidx];
#pragma unroll
                for (int q = 0; q < 4; ++q) cmac(acc[k][q], m, x[q]);
            }
        }
    }
    cx* o = out + (size_t)bp * R2 * A.nc + col0;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const int t = tg + k * TG;
        if (t < R2)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (cg + 8 * q < ncol) o[(int64_t)t * A.nc + cg + 8 * q] = acc[k][q];
    }
}

// u[pt + N col] += sum over the ring's boxes of
//   uph[box][pt] sum_{t1,t2} lw[o1][t1] lw[o2][t2] Lambda^L[box][leaf(pt)][t][col]
// CTA = (leaf, PB x PB block of its points, rhs tile).  The twelve boxes'
// leaf tiles stream through a double buffer of asynchronous copies; per box
// the o2 interpolation is applied once per (o2, t1, col) and reused by every
// row o1 of the block (separable Lagrange weights).
template <typename Real, int RP, int PB>
__global__ void __launch_bounds__(256) k2_term(const RingArgs A, const typename C2D<Real>::T* __restrict__ uph,
                                               const Real* __restrict__ lw,
                                               const typename C2D<Real>::T* __restrict__ lam,
                                               typename C2D<Real>::T* __restrict__ u, int rt)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP, PAD = 16 / PB, KMAX = PB * PB * 32 / 256;
    extern __shared__ __align__(16) unsigned char sraw[];
    cx* Ls = reinterpret_cast<cx*>(sraw);      // [2][R2][rt]
    const int SS = RP * rt + PAD;                // stride of one o2 in Ss
    cx* Ss = Ls + 2 * R2 * rt;                   // [PB][RP][rt] (+ pad per o2)
    cx* Us = Ss + PB * SS;                       // [2][PB * PB] uph of the block
    cx* W1 = Us + 2 * PB * PB;   // [PB][RP] Lagrange weights of the block's rows, as (w, w) pairs
    cx* W2 = W1 + PB * RP;       // [PB][RP] the same for its columns
    const int64_t N = (int64_t)A.n * A.n, mm = (int64_t)A.m * A.m;
    const int K = A.n / A.m, nb1 = K / PB;
    const int ntile = (A.nc + rt - 1) / rt;
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t rest = blockIdx.x / ntile;
    const int pb = (int)(rest % (nb1 * nb1));
    const int64_t leaf = rest / (nb1 * nb1);
    const int o1b = (pb / nb1) * PB, o2b = (pb % nb1) * PB;
    const int64_t n1b = (leaf / A.m) * K + o1b, n2b = (leaf % A.m) * K + o2b;
    const int col0 = tile * rt, ncol = min(rt, A.nc - col0);
    for (int e = threadIdx.x; e < PB * RP; e += blockDim.x) {
        const Real w1 = lw[(o1b + e / RP) * RP + e % RP], w2 = lw[(o2b + e / RP) * RP + e % RP];
        W1[e].x = W1[e].y = w1;
        W2[e].x = W2[e].y = w2;
    }
    auto issue = [&](int b) {
        const cx* lb = lam + ((size_t)(b * mm + leaf) * R2) * A.nc + col0;
        cx* ld = Ls + (b & 1) * R2 * rt;
        for (int e = threadIdx.x; e < R2 * rt; e += blockDim.x) {
            const int t = e / rt, cl = e % rt;
            cp_async_cx(ld + e, cl < ncol ? lb + (int64_t)t * A.nc + cl : lb, cl < ncol);
        }
        for (int e = threadIdx.x; e < PB * PB; e += blockDim.x)
            cp_async_cx(Us + (b & 1) * PB * PB + e, uph + b * N + (n1b + e / PB) * A.n + n2b + e % PB, true);
        asm volatile("cp.async.commit_group;\n" ::);
    };
    cx acc[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) acc[k] = zc<cx>();
    issue(0);
    for (int b = 0; b < 12; ++b) {
        if (b + 1 < 12) {
            issue(b + 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const cx* Lb = Ls + (b & 1) * R2 * rt;
        const cx* Ub = Us + (b & 1) * PB * PB;
        // S[o2][t1][col] = sum_t2 w2[o2][t2] Lambda[t1 RP + t2][col]
        for (int e = threadIdx.x; e < PB * RP * rt; e += blockDim.x) {
            const int cl = e % rt, t1 = (e / rt) % RP, o2 = e / (rt * RP);
            const cx* lr = Lb + t1 * RP * rt + cl;
            cx sv = zc<cx>();
#pragma unroll
            for (int t2 = 0; t2 < RP; ++t2) sv = p2fma(W2[o2 * RP + t2], lr[t2 * rt], sv);
            Ss[o2 * SS + t1 * rt + cl] = sv;
        }
        __syncthreads();
        // acc(o1, o2, col) += uph * sum_t1 w1[o1][t1] S[o2][t1][col]
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int q = threadIdx.x + k * 256;
            if (q < PB * PB * rt) {
                const int o2 = q % PB, cl = (q / PB) % rt, o1 = q / (PB * rt);
                const cx* sr = Ss + o2 * SS + cl;
                cx v = zc<cx>();
#pragma unroll
                for (int t1 = 0; t1 < RP; ++t1) v = p2fma(W1[o1 * RP + t1], sr[t1 * rt], v);
                cmac(acc[k], Ub[o1 * PB + o2], v);
            }
        }
        __syncthreads();   // buffers of box b and Ss are free again
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int q = threadIdx.x + k * 256;
        if (q < PB * PB * rt) {
            const int o2 = q % PB, cl = (q / PB) % rt, o1 = q / (PB * rt);
            if (cl < ncol) {
                cx* up = u + (n1b + o1) * A.n + n2b + o2 + N * (col0 + cl);
                cx o = *up;
                addc(o, acc[k]);
                *up = o;
            }
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Adjoint of the termination: for box b and leaf (PB-free form),
//   Lambda^L[b][leaf][t1 RP + t2][col] = sum over the leaf's K x K points of
//   conj(uph[b][pt]) lw[o1][t1] lw[o2][t2] y[pt][col].
// CTA = (box, leaf, rhs tile); the leaf's points stream in chunks of RC rows
// (RC K <= 64 points); per chunk the o2 weights are applied once per
// (row, t2, col), then the o1 weights accumulate into registers.
template <typename Real, int RP>
__global__ void __launch_bounds__(256) k2_term_adj(const RingArgs A, const typename C2D<Real>::T* __restrict__ uph,
                                                   const Real* __restrict__ lw,
                                                   const typename C2D<Real>::T* __restrict__ y,
                                                   typename C2D<Real>::T* __restrict__ lam, int rt)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP, KA = (R2 * 32 + 255) / 256;
    extern __shared__ __align__(16) unsigned char sraw[];
    const int K = A.n / A.m;
    const int RC = min(K, max(1, 64 / K));
    const int YS = rt + 1;                               // padded point stride
    cx* Ys = reinterpret_cast<cx*>(sraw);                // [RC K <= max(64, K)][YS]
    cx* Ss = Ys + max(64, K) * YS;                       // [RC <= 8][RP][rt]
    Real* Wl = reinterpret_cast<Real*>(Ss + 8 * RP * rt);   // [K][RP]
    const int64_t N = (int64_t)A.n * A.n, mm = (int64_t)A.m * A.m;
    const int ntile = (A.nc + rt - 1) / rt;
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t rest = blockIdx.x / ntile;
    const int64_t leaf = rest % mm;
    const int b = (int)(rest / mm);
    const int64_t n1b = (leaf / A.m) * K, n2b = (leaf % A.m) * K;
    const int col0 = tile * rt, ncol = min(rt, A.nc - col0);
    for (int e = threadIdx.x; e < K * RP; e += blockDim.x) Wl[e] = lw[e];
    cx acc[KA];
#pragma unroll
    for (int k = 0; k < KA; ++k) acc[k] = zc<cx>();
    for (int r0 = 0; r0 < K; r0 += RC) {
        __syncthreads();
        const int np = RC * K;
        for (int e = threadIdx.x; e < np * rt; e += blockDim.x) {
            const int pidx = e % np, cl = e / np;
            const int64_t pt = (n1b + r0 + pidx / K) * A.n + n2b + pidx % K;
            cx v = zc<cx>();
            if (cl < ncol) {
                cx w = uph[b * N + pt];
                w.y = -w.y;
                v = mulc(w, y[pt + N * (col0 + cl)]);
            }
            Ys[pidx * YS + cl] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < RC * RP * rt; e += blockDim.x) {
            const int cl = e % rt, t2 = (e / rt) % RP, row = e / (rt * RP);
            const cx* yr = Ys + (row * K) * YS + cl;
            cx sv = zc<cx>();
            for (int o2 = 0; o2 < K; ++o2) {
                const Real w = Wl[o2 * RP + t2];
                const cx x = yr[o2 * YS];
                sv.x += w * x.x;
                sv.y += w * x.y;
            }
            Ss[(row * RP + t2) * rt + cl] = sv;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KA; ++k) {
            const int q = threadIdx.x + k * 256;
            if (q < R2 * rt) {
                const int cl = q % rt, t = q / rt, t1 = t / RP, t2 = t % RP;
                for (int row = 0; row < RC; ++row) {
                    const Real w = Wl[(r0 + row) * RP + t1];
                    const cx x = Ss[(row * RP + t2) * rt + cl];
                    acc[k].x += w * x.x;
                    acc[k].y += w * x.y;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < KA; ++k) {
        const int q = threadIdx.x + k * 256;
        if (q < R2 * rt) {
            const int cl = q % rt, t = q / rt;
            if (cl < ncol) lam[((size_t)(b * mm + leaf) * R2 + t) * A.nc + col0 + cl] = acc[k];
        }
    }
}

// Adjoint of Lambda^0 = V' g: g(q_box + leaf) = sum_s conj(V[box][leaf][s]) Lambda^0[box][leaf][s]
// (the boxes of a ring cover disjoint frequencies, so every g entry is written once)
template <typename Real>
__global__ void k2_init_adj(const RingArgs A, int r2, const typename C2D<Real>::T* __restrict__ V,
                            const typename C2D<Real>::T* __restrict__ lam, typename C2D<Real>::T* __restrict__ g)
{
    typedef typename C2D<Real>::T cx;
    const int64_t mm = (int64_t)A.m * A.m, N = (int64_t)A.n * A.n;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 12 * mm * A.nc) return;
    // columns fastest: the r^2 reads of Lambda^0 are coalesced across the warp
    const int col = (int)(e % A.nc);
    const int64_t leaf = (e / A.nc) % mm;
    const int b = (int)(e / ((int64_t)A.nc * mm));
    const cx* vr = V + b * A.v_stride + leaf * r2;
    const cx* lr = lam + ((size_t)(b * mm + leaf) * r2) * A.nc + col;
    cx acc = zc<cx>();
    for (int s2 = 0; s2 < r2; ++s2) {
        cx v = vr[s2];
        v.y = -v.y;
        cmac(acc, v, lr[(int64_t)s2 * A.nc]);
    }
    const int64_t a1 = (int64_t)(A.q1[b] + 0.5 * A.n) + (leaf >> A.Lq);
    const int64_t a2 = (int64_t)(A.q2[b] + 0.5 * A.n) + (leaf & (A.m - 1));
    g[a1 * A.n + a2 + N * col] = acc;
}

// Adjoint of the centre sum, part 1: for each chunk of 1024 points,
//   part[chunk][k][col] = sum_pt conj(KC[pt][k]) y[pt][col];
// thread k keeps all rt columns of its centre frequency.
template <typename Real>
__global__ void __launch_bounds__(256) k2_center_adj_part(const typename C2D<Real>::T* __restrict__ KC,
                                                          const typename C2D<Real>::T* __restrict__ y,
                                                          typename C2D<Real>::T* __restrict__ part, int n, int cc,
                                                          int nc, int rt)
{
    typedef typename C2D<Real>::T cx;
    constexpr int CH = 1024, SUB = 16;
    extern __shared__ __align__(16) unsigned char sraw[];
    cx* Ks = reinterpret_cast<cx*>(sraw);   // [SUB][cc]
    cx* Ys = Ks + SUB * cc;                   // [SUB][rt]
    const int64_t N = (int64_t)n * n;
    const int ntile = (nc + rt - 1) / rt;
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t chunk = blockIdx.x / ntile;
    const int col0 = tile * rt, ncol = min(rt, nc - col0);
    cx acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = zc<cx>();
    const int k = threadIdx.x;
    for (int p0 = 0; p0 < CH; p0 += SUB) {
        __syncthreads();
        const int64_t pt0 = chunk * CH + p0;
        for (int e = threadIdx.x; e < SUB * cc; e += blockDim.x) Ks[e] = KC[pt0 * cc + e];
        for (int e = threadIdx.x; e < SUB * rt; e += blockDim.x) {
            const int pp = e % SUB, c = e / SUB;
            Ys[pp * rt + c] = c < ncol ? y[pt0 + pp + N * (col0 + c)] : zc<cx>();
        }
        __syncthreads();
        if (k < cc)
            for (int pp = 0; pp < SUB; ++pp) {
                cx kv = Ks[pp * cc + k];
                kv.y = -kv.y;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < rt) cmac(acc[c], kv, Ys[pp * rt + c]);
            }
    }
    if (k < cc)
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (c < ncol) part[(chunk * cc + k) * nc + col0 + c] = acc[c];
}

// part 2: g(centre frequency k)[col] = sum over chunks of part[chunk][k][col]
template <typename Real>
__global__ void k2_center_adj_sum(const typename C2D<Real>::T* __restrict__ part, typename C2D<Real>::T* __restrict__ g,
                                  int n, int csd, int nc, int64_t nchunk)
{
    typedef typename C2D<Real>::T cx;
    const int cc = csd * csd;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)cc * nc) return;
    const int k = (int)(e % cc), col = (int)(e / cc);
    cx acc = zc<cx>();
    for (int64_t ch = 0; ch < nchunk; ++ch) addc(acc, part[(ch * cc + k) * nc + col]);
    const int a1 = k / csd + n / 2 - csd / 2, a2 = k % csd + n / 2 - csd / 2;
    g[(int64_t)a1 * n + a2 + (int64_t)n * n * col] = acc;
}

template <typename Real, int RP>
static EO2<Real, RP> make_eo2(const ibf_plan* p)
{
    EO2<Real, RP> W;
    {
        constexpr int HQ = EO2<Real, RP>::HQ;
        const auto& T0 = p->T[0];
        auto pr = [](double v) {
            typename C2D<Real>::T q;
            q.x = q.y = (Real)v;
            return q;
        };
        for (int t = 0; t < HQ; ++t)
            for (int s = 0; s < RP; ++s) {
                W.PmT[s][t] = pr((T0[t][s] + T0[RP - 1 - t][s]) / 2);
                W.QmT[s][t] = pr((T0[t][s] - T0[RP - 1 - t][s]) / 2);
            }
        if (RP & 1)
            for (int s = 0; s < RP; ++s) W.PmT[s][HQ] = pr(T0[HQ][s]);
        for (int t = 0; t < RP; ++t) {
            for (int s = 0; s < HQ; ++s) {
                W.E[t][s] = pr((T0[s][t] + T0[RP - 1 - s][t]) / 2);
                W.F[t][s] = pr((T0[s][t] - T0[RP - 1 - s][t]) / 2);
            }
            if (RP & 1) W.E[t][HQ] = pr(T0[HQ][t]);
        }
    }
    return W;
}

template <typename Real, int RP>
static int apply_2d_t(ibf_plan* p, const void* gv, void* uv, int nrhs, cudaStream_t st)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP;
    Plan2D* P = (Plan2D*)p->p2d;
    const EO2<Real, RP> W = make_eo2<Real, RP>(p);
    const int64_t N = (int64_t)P->n * P->n;
    static bool attr = false;
    if (!attr) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k2_level_h<Real, RP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_level_g<Real, RP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_switch<Real, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_center<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_term<Real, RP, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_term<Real, RP, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        attr = true;
    }
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        const int nc = std::min(p->max_nrhs, nrhs - c0);
        const cx* g = (const cx*)gv + N * c0;
        cx* u = (cx*)uv + N * c0;
        prof_start(p, st);
        {
            int rtc = 1;
            while (rtc < 32 && rtc < nc) rtc *= 2;
            const size_t smem_c = ((size_t)P->center * P->center * rtc + 128 * 33) * sizeof(cx);
            k2_center<Real><<<(unsigned)(N / 128 * ((nc + rtc - 1) / rtc)), 256, smem_c, st>>>(
                (const cx*)P->KC, g, u, P->n, P->center, nc, rtc);
        }
        prof_mark(p, st, IBF_K_2D);
        // level kernels: rhs tile a power of two, 16 columns (8 in FP64)
        int rt2 = 1, lrt2 = 0;
        while (rt2 < (sizeof(Real) == 8 ? 8 : 16) && rt2 < nc) rt2 *= 2, ++lrt2;   // lthreads <= the bound
        const int lthreads = (2 * RP * rt2 + 31) / 32 * 32;
        const size_t smem_l = (8 * (size_t)R2 * rt2 + 16 * R2) * sizeof(cx);
        const size_t smem_l1 = smem_l + (4 * (size_t)R2 + 4 * rt2) * sizeof(cx);   // + V rows and g of level 1
        // switch and term: rhs tile a power of two up to 32 (it divides 256)
        int rts = 1;
        while (rts < 32 && rts < nc) rts *= 2;
        const int ntile_s = (nc + rts - 1) / rts;
        const size_t smem_s = ((size_t)R2 * R2 + (size_t)R2 * 32) * sizeof(cx);
        auto term_smem = [&](int pbs) {
            return (2 * (size_t)R2 * rts + (size_t)pbs * (RP * rts + 16 / pbs) + 2 * pbs * pbs + 2 * pbs * RP) *
                   sizeof(cx);
        };
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
            const int64_t blocks2 = 12 * (mm / 4) * ((nc + rt2 - 1) / rt2);
            for (int l = 1; l <= R.Lq; ++l) {
                if (l <= R.hq)
                    k2_level_h<Real, RP, false><<<(unsigned)blocks2, lthreads, l == 1 ? smem_l1 : smem_l, st>>>(
                        W, A, l, (const cx*)R.D[l], a, b, rt2, lrt2, l == 1 ? g : nullptr, (const cx*)R.V);
                else
                    k2_level_g<Real, RP, false><<<(unsigned)blocks2, lthreads, smem_l, st>>>(W, A, l, (const cx*)R.D[l], a, b,
                                                                                       rt2, lrt2);
                prof_mark(p, st, IBF_K_2D);
                std::swap(a, b);
                if (l == R.hq) {
                    k2_switch<Real, RP><<<(unsigned)(12 * mm * ((nc + 31) / 32)), 128, smem_s, st>>>(
                        A, (const cx*)R.M, a, b);
                    prof_mark(p, st, IBF_K_2D);
                    std::swap(a, b);
                }
            }
            if (P->n / R.m >= 8)
                k2_term<Real, RP, 8><<<(unsigned)(mm * (P->n / R.m / 8) * (P->n / R.m / 8) * ntile_s), 256,
                                       term_smem(8), st>>>(A, (const cx*)R.uph, (const Real*)R.lw, a, u, rts);
            else
                k2_term<Real, RP, 4><<<(unsigned)(mm * (P->n / R.m / 4) * (P->n / R.m / 4) * ntile_s), 256,
                                       term_smem(4), st>>>(A, (const cx*)R.uph, (const Real*)R.lw, a, u, rts);
            prof_mark(p, st, IBF_K_2D);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "2D apply launch");
}

// g = K^* y: per column slice the centre's adjoint sum, then per ring the
// adjoint steps in reverse order -- termination, G levels Lq..hq+1 (H-form
// kernels with roles swapped), switch, H levels hq..1 (G-form kernels), and
// the V' g adjoint, which writes the ring's own frequencies of g.
template <typename Real, int RP>
static int apply_2d_adj_t(ibf_plan* p, const void* yv, void* gv, int nrhs, cudaStream_t st)
{
    typedef typename C2D<Real>::T cx;
    constexpr int R2 = RP * RP;
    Plan2D* P = (Plan2D*)p->p2d;
    const EO2<Real, RP> W = make_eo2<Real, RP>(p);
    const int64_t N = (int64_t)P->n * P->n;
    static bool attr = false;
    if (!attr) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(k2_level_h<Real, RP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_level_g<Real, RP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_switch<Real, RP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_term_adj<Real, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k2_center_adj_part<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        attr = true;
    }
    const int cc = P->center * P->center;
    if (cc > 256) return set_error(IBF_ERR_UNSUPPORTED, "2D adjoint: centre side above 16");
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        const int nc = std::min(p->max_nrhs, nrhs - c0);
        const cx* y = (const cx*)yv + N * c0;
        cx* g = (cx*)gv + N * c0;
        prof_start(p, st);
        int rts = 1;
        while (rts < 32 && rts < nc) rts *= 2;
        const int ntile_s = (nc + rts - 1) / rts;
        {
            // centre: partial sums per 1024 points into the ring workspace, then their sum
            const int64_t nchunk = N / 1024;
            const size_t smem_c = ((size_t)16 * cc + 16 * rts) * sizeof(cx);
            k2_center_adj_part<Real><<<(unsigned)(nchunk * ntile_s), 256, smem_c, st>>>(
                (const cx*)P->KC, y, (cx*)P->ws[0], P->n, cc, nc, rts);
            k2_center_adj_sum<Real><<<(unsigned)((cc * nc + 255) / 256), 256, 0, st>>>((const cx*)P->ws[0], g, P->n,
                                                                                      P->center, nc, nchunk);
            prof_mark(p, st, IBF_K_2D);
        }
        int rt2 = 1, lrt2 = 0;
        while (rt2 < (sizeof(Real) == 8 ? 8 : 16) && rt2 < nc) rt2 *= 2, ++lrt2;
        const int lthreads = (2 * RP * rt2 + 31) / 32 * 32;
        const size_t smem_l = (8 * (size_t)R2 * rt2 + 16 * R2) * sizeof(cx);
        const size_t smem_s = ((size_t)R2 * R2 + (size_t)R2 * 32) * sizeof(cx);
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
            const int K = P->n / R.m;
            cx* a = (cx*)P->ws[0];
            cx* b = (cx*)P->ws[1];
            const size_t smem_t = ((size_t)std::max(64, K) * (rts + 1) + 8 * RP * rts) * sizeof(cx) +
                                  (size_t)K * RP * sizeof(Real);
            k2_term_adj<Real, RP><<<(unsigned)(12 * mm * ntile_s), 256, smem_t, st>>>(A, (const cx*)R.uph,
                                                                                    (const Real*)R.lw, y, a, rts);
            prof_mark(p, st, IBF_K_2D);
            const int64_t blocks2 = 12 * (mm / 4) * ((nc + rt2 - 1) / rt2);
            auto switch_adj = [&]() {
                k2_switch<Real, RP, true><<<(unsigned)(12 * mm * ((nc + 31) / 32)), 128, smem_s, st>>>(
                    A, (const cx*)R.M, a, b);
                prof_mark(p, st, IBF_K_2D);
                std::swap(a, b);
            };
            if (R.hq == R.Lq) switch_adj();   // forward: the switch follows the last level
            for (int l = R.Lq; l >= 1; --l) {
                if (l > R.hq)
                    k2_level_h<Real, RP, true><<<(unsigned)blocks2, lthreads, smem_l, st>>>(
                        W, A, l, (const cx*)R.D[l], a, b, rt2, lrt2, nullptr, nullptr);
                else
                    k2_level_g<Real, RP, true><<<(unsigned)blocks2, lthreads, smem_l, st>>>(
                        W, A, l, (const cx*)R.D[l], a, b, rt2, lrt2);
                prof_mark(p, st, IBF_K_2D);
                std::swap(a, b);
                if (l == R.hq + 1) switch_adj();   // forward: the switch sits between levels hq and hq+1
            }
            k2_init_adj<Real><<<(unsigned)((12 * mm * nc + 255) / 256), 256, 0, st>>>(A, R2, (const cx*)R.V, a, g);
            prof_mark(p, st, IBF_K_2D);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "2D adjoint launch");
}

int apply_2d_adjoint(ibf_plan* p, const void* y, void* g, int nrhs, cudaStream_t st)
{
    const bool d = p->dtype == IBF_C128;
    switch (p->r) {
    case 5: return d ? apply_2d_adj_t<double, 5>(p, y, g, nrhs, st) : apply_2d_adj_t<float, 5>(p, y, g, nrhs, st);
    case 7: return d ? apply_2d_adj_t<double, 7>(p, y, g, nrhs, st) : apply_2d_adj_t<float, 7>(p, y, g, nrhs, st);
    case 9: return d ? apply_2d_adj_t<double, 9>(p, y, g, nrhs, st) : apply_2d_adj_t<float, 9>(p, y, g, nrhs, st);
    default: return set_error(IBF_ERR_UNSUPPORTED, "2D: r must be 5, 7 or 9");
    }
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
    for (const Ring2D& R : P->rings) n += R.Lq + 2;
    return n;
}

}  // namespace ibf
