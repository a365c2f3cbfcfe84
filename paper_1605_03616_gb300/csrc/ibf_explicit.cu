// Explicit-form apply of the preliminary IBF (Sec. 3): the plain form.
//
// u = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^1)^* (V^0)^* g, one kernel per
// factor.  Lambda^l_{i,j} (r complex per box pair and right-hand side) is kept
// in i-major pair order p = i 2^(L-l) + j at every level, element
// (p r + t) nc + col, so the switch's reordering (Sec. 3, step 4) is only a
// change of index arithmetic.  Each butterfly block maps
// Lambda^{l-1}_{i/2, 2j+c} to Lambda^l_{i,j} (eqs. PIBF2, PIBF3).
//
// The optimal form runs the same kernels with its compressed blocks: rank r0
// at every level after the sweep-out stage, and after the sweep-in stage a
// rank per level (r_out x r_in blocks, an r_g x r_h middle factor).
#include <algorithm>

#include "ibf_internal.h"

namespace ibf {

// Kernels are templates on the complex type: double2 for FP64 plans, float2
// for FP32 plans (factors built in FP64, then stored in FP32).
template <typename cx> struct RealOf;
template <> struct RealOf<double2> { typedef double T; };
template <> struct RealOf<float2> { typedef float T; };

template <typename cx>
__device__ __forceinline__ cx cmk(typename RealOf<cx>::T re, typename RealOf<cx>::T im)
{
    cx o;
    o.x = re;
    o.y = im;
    return o;
}
template <typename cx>
__device__ __forceinline__ cx cmul(cx a, cx b) { return cmk<cx>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename cx>
__device__ __forceinline__ cx cmulc(cx a, cx b)  // conj(a) * b
{
    return cmk<cx>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename cx>
__device__ __forceinline__ void cadd(cx& a, cx b) { a.x += b.x; a.y += b.y; }

// Lambda^0[k][t][col] = V[k][t] g[k + N col]       ((V^0)^* g, eq. step2mv1)
template <typename cd>
__global__ void kx_init(const cd* V, const cd* g, cd* lam, int64_t N, int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * r * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % r);
    int64_t k = e / ((int64_t)nc * r);
    lam[e] = cmul(V[k * r + t], g[k + N * col]);
}

// g[k + N col] = sum_t conj(V[k][t]) Lambda^0[k][t][col]
template <typename cd>
__global__ void kx_init_adj(const cd* V, const cd* lam, cd* g, int64_t N, int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * nc) return;
    int64_t k = e % N;
    int col = (int)(e / N);
    cd acc = cmk<cd>(0, 0);
    for (int t = 0; t < r; ++t) cadd(acc, cmulc(V[k * r + t], lam[(k * r + t) * nc + col]));
    g[k + N * col] = acc;
}

// one butterfly level l: out pair p = (i,j) (rank ro) from in pairs
// (i/2, 2j+c) (rank ri) through the ro x ri blocks blk[p][c]
template <typename cd>
__global__ void kx_level(const cd* blk, const cd* in, cd* out, int L, int l, int ro, int ri, int nc, int64_t N)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * ro * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % ro);
    int64_t p = e / ((int64_t)nc * ro);
    int64_t nj = 1LL << (L - l);
    int64_t i = p >> (L - l), j = p & (nj - 1);
    int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
    cd acc = cmk<cd>(0, 0);
    for (int c = 0; c < 2; ++c) {
        const cd* row = blk + ((p * 2 + c) * ro + t) * ri;
        const cd* v = in + (q0 + c) * ri * nc + col;
        for (int s = 0; s < ri; ++s) cadd(acc, cmul(row[s], v[(int64_t)s * nc]));
    }
    out[e] = acc;
}

// adjoint of level l: in pair q = (i', C) at level l-1 gathers from the two
// out pairs (2i'+a, C/2) at level l with the conjugated blocks
template <typename cd>
__global__ void kx_level_adj(const cd* blk, const cd* out, cd* in, int L, int l, int ro, int ri, int nc,
                             int64_t N)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * ri * nc) return;
    int col = (int)(e % nc);
    int s = (int)((e / nc) % ri);
    int64_t q = e / ((int64_t)nc * ri);
    int64_t nC = 1LL << (L - l + 1), nj = nC >> 1;
    int64_t ip = q >> (L - l + 1), C = q & (nC - 1);
    int64_t j = C >> 1;
    int c = (int)(C & 1);
    cd acc = cmk<cd>(0, 0);
    for (int a = 0; a < 2; ++a) {
        int64_t p = (2 * ip + a) * nj + j;
        const cd* col_blk = blk + ((p * 2 + c) * ro) * ri + s;
        const cd* v = out + p * ro * nc + col;
        for (int t = 0; t < ro; ++t) cadd(acc, cmulc(col_blk[(int64_t)t * ri], v[(int64_t)t * nc]));
    }
    in[e] = acc;
}

// Warp-per-pair forms of the two level kernels above (same arithmetic, same
// outputs).  A level streams its blocks once (2 ro ri entries per pair) and
// reads two contiguous input pairs, so it should run at the HBM rate; one
// thread per output entry instead issues ri dependent loads per block row
// and stays latency-bound.  Here one warp owns one output pair: it copies the
// pair's blocks and, per tile of kXCT columns, its inputs into a shared-memory
// slice with asynchronous copies (every lane several in flight), then each
// lane computes outputs (t, col) of the tile from shared memory (block rows
// read as broadcasts, inputs by consecutive columns) and stores them
// coalesced.  Ranks up to kXRmax.
constexpr int kXWarps = 8;     // warps (pairs) per CTA
constexpr int kXCT = 8;        // columns per tile
constexpr int kXRmax = 16;

__device__ __forceinline__ void xcp(float2* d, const float2* s)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(s)
                 : "memory");
}
__device__ __forceinline__ void xcp(double2* d, const double2* s)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(s)
                 : "memory");
}
__device__ __forceinline__ void xcp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// shared memory per warp: the two blocks (or the two gathered blocks of the
// adjoint) and one tile of two input pairs
template <typename cd>
constexpr size_t xslice_elems() { return 2 * kXRmax * kXRmax + 2 * kXRmax * kXCT; }

template <typename cd>
__global__ void __launch_bounds__(kXWarps * 32) kx_level_w(const cd* blk, const cd* in, cd* out, int L, int l, int ro,
                                                            int ri, int nc, int64_t N)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kXWarps + w;
    if (p >= N) return;
    cd* sb = reinterpret_cast<cd*>(xsm) + w * xslice_elems<cd>();   // [c][t][s]
    cd* sx = sb + 2 * kXRmax * kXRmax;                                // [c][s][col of tile]
    const int64_t nj = 1LL << (L - l);
    const int64_t i = p >> (L - l), j = p & (nj - 1);
    const int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
    const cd* bp = blk + p * 2 * ro * ri;
    const int nb = 2 * ro * ri;
    for (int e = lane; e < nb; e += 32) xcp(sb + e, bp + e);
    for (int c0 = 0; c0 < nc; c0 += kXCT) {
        const int nt = min(kXCT, nc - c0);
        const cd* xin = in + q0 * ri * nc + c0;
        for (int e = lane; e < 2 * ri * nt; e += 32) {
            const int cs = e / nt, col = e - cs * nt;   // cs = c ri + s
            xcp(sx + cs * kXCT + col, xin + (int64_t)cs * nc + col);
        }
        xcp_wait();
        __syncwarp();
        for (int o = lane; o < ro * nt; o += 32) {
            const int t = o / nt, col = o - t * nt;
            cd acc = cmk<cd>(0, 0);
            for (int c = 0; c < 2; ++c) {
                const cd* row = sb + (c * ro + t) * ri;
                const cd* v = sx + c * ri * kXCT + col;
#pragma unroll 4
                for (int s2 = 0; s2 < ri; ++s2) cadd(acc, cmul(row[s2], v[s2 * kXCT]));
            }
            out[(p * ro + t) * nc + c0 + col] = acc;
        }
        __syncwarp();   // the tile's inputs are read before the next tile's copies
    }
}

// Persistent, double-buffered form of kx_level_w for nc <= kXPipeCols: every
// warp walks pairs w, w + W, w + 2W, ... (W = warps in the grid) with two
// shared-memory slices sized to the level's ranks (2 ro ri + 2 ri nc
// elements), and issues the copies of its next pair before computing the
// current one, so copies stay in flight through the arithmetic.
constexpr int kXPipeCols = 16;
constexpr int kXMinCols = 4;   // fewer columns leave most lanes of a pair's warp idle

template <typename cd>
__global__ void __launch_bounds__(kXWarps * 32) kx_level_wp(const cd* blk, const cd* in, cd* out, int L, int l, int ro,
                                                             int ri, int nc, int64_t N, int slice)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * kXWarps;
    cd* s0 = reinterpret_cast<cd*>(xsm) + (size_t)w * 2 * slice;
    cd* s1 = s0 + slice;
    const int nb = 2 * ro * ri, nx = 2 * ri * nc;
    const int64_t nj = 1LL << (L - l);
    auto issue = [&](int64_t p, cd* sl) {
        const int64_t i = p >> (L - l), j = p & (nj - 1);
        const int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
        const cd* bp = blk + p * nb;
        const cd* xp = in + q0 * ri * nc;          // the two input pairs are contiguous
        for (int e = lane; e < nb; e += 32) xcp(sl + e, bp + e);
        for (int e = lane; e < nx; e += 32) xcp(sl + nb + e, xp + e);
    };
    int64_t p = (int64_t)blockIdx.x * kXWarps + w;
    if (p < N) issue(p, s0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int it = 0; p < N; ++it, p += W) {
        cd* cur = (it & 1) ? s1 : s0;
        if (p + W < N) issue(p + W, (it & 1) ? s0 : s1);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncwarp();
        const cd* sx = cur + nb;                   // [c][s][col]
        for (int o = lane; o < ro * nc; o += 32) {
            const int t = o / nc, col = o - t * nc;
            cd acc = cmk<cd>(0, 0);
            for (int c = 0; c < 2; ++c) {
                const cd* row = cur + (c * ro + t) * ri;
                const cd* v = sx + c * ri * nc + col;
#pragma unroll 4
                for (int s2 = 0; s2 < ri; ++s2) cadd(acc, cmul(row[s2], v[s2 * nc]));
            }
            out[(p * ro + t) * nc + col] = acc;
        }
        __syncwarp();   // every lane is done with this slice before it is refilled
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// adjoint of level l, warp per input pair q = (i', C) of level l-1: it
// gathers from the output pairs (2i'+a, C/2), a = 0, 1, through block c = C&1
// of each, conjugate-transposed
template <typename cd>
__global__ void __launch_bounds__(kXWarps * 32) kx_level_adj_w(const cd* blk, const cd* out, cd* in, int L, int l,
                                                                int ro, int ri, int nc, int64_t N)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * kXWarps + w;
    if (q >= N) return;
    cd* sb = reinterpret_cast<cd*>(xsm) + w * xslice_elems<cd>();   // [a][t][s]
    cd* sy = sb + 2 * kXRmax * kXRmax;                                // [a][t][col of tile]
    const int64_t nC = 1LL << (L - l + 1), nj = nC >> 1;
    const int64_t ip = q >> (L - l + 1), C = q & (nC - 1);
    const int64_t j = C >> 1;
    const int c = (int)(C & 1);
    const int nb = ro * ri;
    for (int a = 0; a < 2; ++a) {
        const int64_t pa = (2 * ip + a) * nj + j;
        const cd* bp = blk + (pa * 2 + c) * nb;
        for (int e = lane; e < nb; e += 32) xcp(sb + a * nb + e, bp + e);
    }
    for (int c0 = 0; c0 < nc; c0 += kXCT) {
        const int nt = min(kXCT, nc - c0);
        for (int a = 0; a < 2; ++a) {
            const int64_t pa = (2 * ip + a) * nj + j;
            const cd* yin = out + pa * ro * nc + c0;
            for (int e = lane; e < ro * nt; e += 32) {
                const int t = e / nt, col = e - t * nt;
                xcp(sy + (a * ro + t) * kXCT + col, yin + (int64_t)t * nc + col);
            }
        }
        xcp_wait();
        __syncwarp();
        for (int o = lane; o < ri * nt; o += 32) {
            const int s2 = o / nt, col = o - s2 * nt;
            cd acc = cmk<cd>(0, 0);
            for (int a = 0; a < 2; ++a) {
                const cd* bcol = sb + a * nb + s2;
                const cd* v = sy + a * ro * kXCT + col;
#pragma unroll 4
                for (int t = 0; t < ro; ++t) cadd(acc, cmulc(bcol[t * ri], v[t * kXCT]));
            }
            in[(q * ri + s2) * nc + c0 + col] = acc;
        }
        __syncwarp();
    }
}

// switch at level h: out_p = M~_p in_p (eq. switchlocM), M~_p of rows x cols
// (rank after x rank before the switch), or its adjoint
template <typename cd>
__global__ void kx_switch(const cd* M, const cd* in, cd* out, int rows, int cols, int nc, int64_t N, int adj)
{
    const int rout = adj ? cols : rows, rin = adj ? rows : cols;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * rout * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % rout);
    int64_t p = e / ((int64_t)nc * rout);
    const cd* Mp = M + p * rows * cols;
    const cd* v = in + p * rin * nc + col;
    cd acc = cmk<cd>(0, 0);
    if (!adj)
        for (int s = 0; s < cols; ++s) cadd(acc, cmul(Mp[t * cols + s], v[(int64_t)s * nc]));
    else
        for (int s = 0; s < rows; ++s) cadd(acc, cmulc(Mp[s * cols + t], v[(int64_t)s * nc]));
    out[e] = acc;
}

// u[perm[n] + nx col] = sum_t U[n][t] Lambda^L[leaf(n)][t][col]   (eq. PIBFbf3)
template <typename cd>
__global__ void kx_term(const cd* U, const int32_t* leaf, const int32_t* perm, const cd* lam, cd* u, int64_t nx,
                        int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nx * nc) return;
    int64_t n = e % nx;
    int col = (int)(e / nx);
    const cd* v = lam + (int64_t)leaf[n] * r * nc + col;
    cd acc = cmk<cd>(0, 0);
    for (int t = 0; t < r; ++t) cadd(acc, cmul(U[n * r + t], v[(int64_t)t * nc]));
    u[perm[n] + nx * col] = acc;
}

// Lambda^L[i][t][col] = sum_{n in leaf i} conj(U[n][t]) y[perm[n] + nx col]
template <typename cd>
__global__ void kx_term_adj(const cd* U, const int32_t* off, const int32_t* perm, const cd* y, cd* lam, int64_t N,
                            int64_t nx, int r, int nc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * r * nc) return;
    int col = (int)(e % nc);
    int t = (int)((e / nc) % r);
    int64_t i = e / ((int64_t)nc * r);
    cd acc = cmk<cd>(0, 0);
    for (int32_t n = off[i]; n < off[i + 1]; ++n) cadd(acc, cmulc(U[(int64_t)n * r + t], y[perm[n] + nx * col]));
    lam[e] = acc;
}

static inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// the warp-per-pair level kernels use kXWarps slices of shared memory (96 KB
// for complex128): raise their dynamic shared-memory limit once per device
template <typename cd>
static size_t xlevel_smem()
{
    static bool done[64] = {false};
    const size_t bytes = kXWarps * xslice_elems<cd>() * sizeof(cd);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev]) {
        cudaFuncSetAttribute(kx_level_w<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        cudaFuncSetAttribute(kx_level_adj_w<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    return bytes;
}

// rank of Lambda^l before the switch (H side, l <= h) and after it (G side,
// l >= h)
static inline int rank_h(const ibf_plan* p, int l)
{
    return !p->rk_h.empty() ? p->rk_h[l] : (p->ra > 0 ? p->ra : p->r);
}
static inline int rank_g(const ibf_plan* p, int l)
{
    return !p->rk_g.empty() ? p->rk_g[l] : (p->ra > 0 ? p->ra : p->r);
}
// output and input rank of the butterfly blocks of level l
static inline int rank_out(const ibf_plan* p, int l) { return l <= p->h ? rank_h(p, l) : rank_g(p, l); }
static inline int rank_in(const ibf_plan* p, int l) { return l <= p->h ? rank_h(p, l - 1) : rank_g(p, l - 1); }

int explicit_launches(const ibf_plan* p) { return p->L + 3; }

// persistent warp-per-pair level: as many CTAs as are resident at once;
// false (nothing launched) if its slices do not fit one CTA's shared memory
template <typename cd>
static bool launch_level_wp(const cd* blk, const cd* in, cd* out, int L, int l, int ro, int ri, int nc, int64_t N,
                            cudaStream_t st)
{
    const int slice = (2 * ro * ri + 2 * ri * nc + 1) & ~1;   // even: 16-byte aligned slices for complex64
    const size_t smem = (size_t)kXWarps * 2 * slice * sizeof(cd);
    int dev = 0, nsm = 0, occ = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) return false;
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64 || !done[dev]) {
        cudaFuncSetAttribute(kx_level_wp<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kx_level_wp<cd>, kXWarps * 32, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const int64_t blocks = std::min<int64_t>((N + kXWarps - 1) / kXWarps, (int64_t)nsm * occ);
    kx_level_wp<cd><<<(unsigned)blocks, kXWarps * 32, smem, st>>>(blk, in, out, L, l, ro, ri, nc, N, slice);
    return true;
}

template <typename cd>
static int explicit_apply_t(ibf_plan* p, const void* gv, void* uv, int nrhs, cudaStream_t st)
{
    const int L = p->L, h = p->h;
    const int64_t N = p->N;
    const int k0 = rank_h(p, 0), kL = rank_g(p, L), mr = rank_g(p, h), mc = rank_h(p, h);
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        int nc = std::min(p->max_nrhs, nrhs - c0);
        const cd* g = (const cd*)gv + N * c0;
        cd* u = (cd*)uv + p->nx * c0;
        cd* a = (cd*)p->ws[0];
        cd* b = (cd*)p->ws[1];
        prof_start(p, st);
        kx_init<<<nb(N * k0 * nc), 256, 0, st>>>((const cd*)p->eV, g, a, N, k0, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_INIT);
        for (int l = 1; l <= L; ++l) {
            const int ro = rank_out(p, l), ri = rank_in(p, l);
            // warp per pair where the level is memory-bound (complex64) and the
            // pair has enough outputs for a warp; FP64 levels are bound by the
            // FP64 pipe and keep one thread per output entry
            const bool warp = sizeof(cd) == sizeof(float2) && nc >= kXMinCols;
            if (warp && nc <= kXPipeCols && launch_level_wp<cd>((const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N, st)) {
            } else if (warp && ro <= kXRmax && ri <= kXRmax)
                kx_level_w<cd><<<(unsigned)((N + kXWarps - 1) / kXWarps), kXWarps * 32, xlevel_smem<cd>(), st>>>(
                    (const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            else
                kx_level<<<nb(N * ro * nc), 256, 0, st>>>((const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            prof_mark(p, st, IBF_K_EXPLICIT_LEVEL);
            std::swap(a, b);
            if (l == h) {
                kx_switch<<<nb(N * mr * nc), 256, 0, st>>>((const cd*)p->eM, a, b, mr, mc, nc, N, 0);
                prof_mark(p, st, IBF_K_EXPLICIT_SWITCH);
                std::swap(a, b);
            }
        }
        kx_term<<<nb(p->nx * nc), 256, 0, st>>>((const cd*)p->eU, p->d_leaf, p->d_perm, a, u, p->nx, kL, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_TERM);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "explicit apply launch");
}

template <typename cd>
static int explicit_adjoint_t(ibf_plan* p, const void* yv, void* gv, int nrhs, cudaStream_t st)
{
    const int L = p->L, h = p->h;
    const int64_t N = p->N;
    const int k0 = rank_h(p, 0), kL = rank_g(p, L), mr = rank_g(p, h), mc = rank_h(p, h);
    for (int c0 = 0; c0 < nrhs; c0 += p->max_nrhs) {
        int nc = std::min(p->max_nrhs, nrhs - c0);
        const cd* y = (const cd*)yv + p->nx * c0;
        cd* g = (cd*)gv + N * c0;
        cd* a = (cd*)p->ws[0];
        cd* b = (cd*)p->ws[1];
        prof_start(p, st);
        kx_term_adj<<<nb(N * kL * nc), 256, 0, st>>>((const cd*)p->eU, p->d_off, p->d_perm, y, a, N, p->nx, kL, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_TERM);
        for (int l = L; l >= 1; --l) {
            if (l == h) {
                kx_switch<<<nb(N * mc * nc), 256, 0, st>>>((const cd*)p->eM, a, b, mr, mc, nc, N, 1);
                prof_mark(p, st, IBF_K_EXPLICIT_SWITCH);
                std::swap(a, b);
            }
            const int ro = rank_out(p, l), ri = rank_in(p, l);
            if (sizeof(cd) == sizeof(float2) && nc >= kXMinCols && ro <= kXRmax && ri <= kXRmax)
                kx_level_adj_w<cd><<<(unsigned)((N + kXWarps - 1) / kXWarps), kXWarps * 32, xlevel_smem<cd>(), st>>>(
                    (const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            else
                kx_level_adj<<<nb(N * ri * nc), 256, 0, st>>>((const cd*)p->eblk[l], a, b, L, l, ro, ri, nc, N);
            prof_mark(p, st, IBF_K_EXPLICIT_LEVEL);
            std::swap(a, b);
        }
        kx_init_adj<<<nb(N * nc), 256, 0, st>>>((const cd*)p->eV, a, g, N, k0, nc);
        prof_mark(p, st, IBF_K_EXPLICIT_INIT);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : cuda_error(e, "explicit adjoint launch");
}

int explicit_apply(ibf_plan* p, const void* gv, void* uv, int nrhs, cudaStream_t st)
{
    return p->dtype == IBF_C128 ? explicit_apply_t<double2>(p, gv, uv, nrhs, st)
                                : explicit_apply_t<float2>(p, gv, uv, nrhs, st);
}

int explicit_adjoint(ibf_plan* p, const void* yv, void* gv, int nrhs, cudaStream_t st)
{
    return p->dtype == IBF_C128 ? explicit_adjoint_t<double2>(p, yv, gv, nrhs, st)
                                : explicit_adjoint_t<float2>(p, yv, gv, nrhs, st);
}

__global__ void kx_demote(const double2* a, float2* b, int64_t n)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// FP32 plans of the explicit and optimal forms: the factors are built (and
// compressed) in FP64, then replaced by complex64 copies.
int explicit_demote(ibf_plan* p, void* (*alloc)(ibf_plan*, size_t), void (*release)(ibf_plan*, void*))
{
    const int L = p->L, h = p->h;
    const int64_t N = p->N;
    auto one = [&](void*& f, int64_t n) -> int {
        void* q = alloc(p, sizeof(float2) * (size_t)n);
        if (!q) return set_error(IBF_ERR_OOM, "FP32 factor copy");
        kx_demote<<<nb(n), 256>>>((const double2*)f, (float2*)q, n);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(e, "FP32 factor copy");
        release(p, f);
        f = q;
        return IBF_OK;
    };
    int rc;
    if ((rc = one(p->eV, N * rank_h(p, 0)))) return rc;
    if ((rc = one(p->eM, N * rank_g(p, h) * rank_h(p, h)))) return rc;
    if ((rc = one(p->eU, p->nx * rank_g(p, L)))) return rc;
    for (int l = 1; l <= L; ++l)
        if ((rc = one(p->eblk[l], N * 2 * rank_out(p, l) * rank_in(p, l)))) return rc;
    p->factor_bytes = sizeof(float2) * (size_t)p->nnz;
    return IBF_OK;
}

}  // namespace ibf
