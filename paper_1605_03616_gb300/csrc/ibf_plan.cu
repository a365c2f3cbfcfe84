// Plan construction for the preliminary IBF (Sec. 3) and the C ABI entry
// points of include/ibf.h.
//
// Every factor entry is a product of phases e(Phi) = exp(2 pi i Phi) and
// Lagrange weights (Sec. 2.1, eqs. ab1/ab2).  Phases are evaluated in FP64 on
// the device; the argument is reduced modulo 1 (an exact subtraction) before
// sincospi, because Phi grows to ~N.  This translation unit is compiled with
// -fmad=false so that box centres, grid points and phases round exactly like
// a plain sequential FP64 evaluation of the paper's formulas.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "ibf_2d.h"
#include "ibf_internal.h"

namespace ibf {

static thread_local int g_last_code = IBF_OK;
static thread_local char g_last_msg[512] = "";

int set_error(int code, const std::string& msg)
{
    g_last_code = code;
    snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg.c_str());
    return code;
}

int cuda_error(cudaError_t e, const char* what)
{
    return set_error(IBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// device geometry (1D): X box (l,i) = [i 2^-l, (i+1) 2^-l),
// Omega box (l,j) = [-N/2 + j N 2^-l, -N/2 + (j+1) N 2^-l); centres are
// midpoints, so the Omega root is centred at 0.
// ---------------------------------------------------------------------------
struct Geo {
    int64_t N;
    int L, r, phase;
    double z[kMaxR];
    int nco;                       // IBF_PHASE_FIO1D_SERIES: terms of c(x)
    double ca[kMaxCoef], cb[kMaxCoef];
};

__device__ __forceinline__ double pow2(int l) { return (double)(1LL << l); }
__device__ __forceinline__ double xc(int l, int64_t i) { return ((double)i + 0.5) / pow2(l); }
__device__ __forceinline__ double xw(int l) { return 1.0 / pow2(l); }
__device__ __forceinline__ double ww(int64_t N, int l) { return (double)N / pow2(l); }
__device__ __forceinline__ double wc(int64_t N, int l, int64_t j) { return -0.5 * (double)N + ((double)j + 0.5) * ww(N, l); }

// Phase functions (Assumption 1.1; Sec. 6.1, 6.2, the 1D FIO with a series
// coefficient, and a separable test phase).
__device__ __forceinline__ double phi(const Geo& G, double x, double xi)
{
    const int ph = G.phase;
    if (ph == IBF_PHASE_NUFFT) return x * xi;
    if (ph == IBF_PHASE_FIO1D) {
        double c = (2.0 + sin(2.0 * 3.141592653589793 * x)) / 8.0;
        return x * xi + c * fabs(xi);
    }
    if (ph == IBF_PHASE_FIO1D_SERIES) {
        // c(x) = sum_m a_m cos(2 pi m x) + b_m sin(2 pi m x), summed in order of m
        double c = 0.0;
        for (int m = 0; m < G.nco; ++m) {
            const double arg = 2.0 * 3.141592653589793 * (double)m * x;
            c += G.ca[m] * cos(arg) + G.cb[m] * sin(arg);
        }
        return x * xi + c * fabs(xi);
    }
    // IBF_PHASE_SEPARABLE
    return 0.75 * sin(2.0 * 3.141592653589793 * x) + (0.125 * fabs(xi) + 0.3 * sin(0.1 * xi));
}

// e(t) = exp(2 pi i t) after removing the nearest integer from t
__device__ __forceinline__ double2 e2pi(double t)
{
    double th = t - rint(t);
    double s, c;
    sincospi(2.0 * th, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double a, double2 b) { return make_double2(a * b.x, a * b.y); }

// Lagrange polynomial M_t on the Chebyshev grid z, product form (Sec. 2.1)
__device__ __forceinline__ double lag(const Geo& G, int t, double u)
{
    double p = 1.0;
    for (int m = 0; m < G.r; ++m)
        if (m != t) p *= (u - G.z[m]) / (G.z[t] - G.z[m]);
    return p;
}

__device__ __forceinline__ double gp(double c, double w, const Geo& G, int t) { return c + w * G.z[t]; }

template <typename C>
__device__ __forceinline__ void store(C* p, double2 v);
template <>
__device__ __forceinline__ void store<double2>(double2* p, double2 v) { *p = v; }
template <>
__device__ __forceinline__ void store<float2>(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

// ---------------------------------------------------------------------------
// explicit factors (complex128), Sec. 3
// ---------------------------------------------------------------------------

// (V^0)^*: column for xi_k; A = root of T_X, B = leaf of xi_k (eq. PIBF1)
__global__ void kE_V(const Geo G, double2* V)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= G.N * G.r) return;
    int t = (int)(e % G.r);
    int64_t k = e / G.r;
    double xi = (double)k - 0.5 * (double)G.N;
    double cA = xc(0, 0), wB = ww(G.N, G.L), cB = wc(G.N, G.L, k);
    double2 v = cmul(e2pi(-phi(G, cA, gp(cB, wB, G, t))), e2pi(phi(G, cA, xi)));
    V[e] = cscale(lag(G, t, (xi - cB) / wB), v);
}

// butterfly blocks of level l: blk[p][c][t][s], p = i 2^(L-l) + j.
// l <= h: eq. PIBF2; l > h: eq. PIBF3.
__global__ void kE_blk(const Geo G, int l, int h, double2* B)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = G.r;
    if (e >= G.N * 2 * r * r) return;
    int s = (int)(e % r);
    int t = (int)((e / r) % r);
    int c = (int)((e / (r * r)) % 2);
    int64_t p = e / (2 * r * r);
    int64_t i = p >> (G.L - l), j = p & ((1LL << (G.L - l)) - 1);
    double cC = wc(G.N, G.L - l + 1, 2 * j + c), wC = ww(G.N, G.L - l + 1);
    double2 v;
    if (l <= h) {
        double cA = xc(l, i);
        double cB = wc(G.N, G.L - l, j), wB = ww(G.N, G.L - l);
        double gCs = gp(cC, wC, G, s);
        v = cscale(lag(G, t, (gCs - cB) / wB),
                   cmul(e2pi(-phi(G, cA, gp(cB, wB, G, t))), e2pi(phi(G, cA, gCs))));
    } else {
        double cA = xc(l, i), wA = xw(l);
        double cP = xc(l - 1, i / 2), wP = xw(l - 1);
        double gAt = gp(cA, wA, G, t);
        v = cscale(lag(G, s, (gAt - cP) / wP),
                   cmul(e2pi(phi(G, gAt, cC)), e2pi(-phi(G, gp(cP, wP, G, s), cC))));
    }
    B[e] = v;
}

// switch blocks M~_{ij}[t][s] = e(Phi(g^A_t, g^B_s)) at level h (eq. switchlocM)
__global__ void kE_M(const Geo G, int h, double2* M)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = G.r;
    if (e >= G.N * r * r) return;
    int s = (int)(e % r);
    int t = (int)((e / r) % r);
    int64_t p = e / (r * r);
    int64_t i = p >> (G.L - h), j = p & ((1LL << (G.L - h)) - 1);
    double cA = xc(h, i), wA = xw(h), cB = wc(G.N, G.L - h, j), wB = ww(G.N, G.L - h);
    M[e] = e2pi(phi(G, gp(cA, wA, G, t), gp(cB, wB, G, s)));
}

// U^L rows for the sorted points (eq. PIBFbf3), B = root of T_Omega
__global__ void kE_U(const Geo G, const double* x, const int32_t* leaf, int64_t nx, double2* U)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nx * G.r) return;
    int t = (int)(e % G.r);
    int64_t n = e / G.r;
    double xn = x[n];
    double cB = wc(G.N, 0, 0), wA = xw(G.L), cA = xc(G.L, leaf[n]);
    double2 v = cmul(e2pi(phi(G, xn, cB)), e2pi(-phi(G, gp(cA, wA, G, t), cB)));
    U[e] = cscale(lag(G, t, (xn - cA) / wA), v);
}

// ---------------------------------------------------------------------------
// structured factors.  Each butterfly block of level l is
//   H: diag(e(-Phi(c_A, g^B_t))) T_c diag(e(Phi(c_A, g^C_s)))          (eq. PIBF2)
//   G: diag(e(Phi(g^A_t, c_C))) T_a^T diag(e(-Phi(g^P_s, c_C)))        (eq. PIBF3)
// The left diagonal of an H level meets the right diagonal of the next level
// on the same grid g^{B^{L-l+1}_C}, so they are stored as one merged phase;
// likewise for the G levels.  The end diagonals merge into V^0, M^h and U^L.
// ---------------------------------------------------------------------------
template <typename C>
__global__ void kS_V(const Geo G, C* V)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= G.N * G.r) return;
    int t = (int)(e % G.r);
    int64_t k = e / G.r;
    double xi = (double)k - 0.5 * (double)G.N;
    double cA = xc(0, 0), wB = ww(G.N, G.L), cB = wc(G.N, G.L, k);
    store(V + e, cscale(lag(G, t, (xi - cB) / wB), e2pi(phi(G, cA, xi))));
}

// H level l (1..h): D[i][C][s], i < 2^l, C < 2^(L-l+1)
template <typename C>
__global__ void kS_Q(const Geo G, int l, C* D)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = G.r;
    const int cb = G.L - l + 1;
    if (e >= (2 * G.N) * r) return;
    int s = (int)(e % r);
    int64_t q = e / r;
    int64_t i = q >> cb, Cc = q & ((1LL << cb) - 1);
    double g = gp(wc(G.N, cb, Cc), ww(G.N, cb), G, s);
    double d = phi(G, xc(l, i), g) - phi(G, xc(l - 1, i / 2), g);
    store(D + e, e2pi(d));
}

// G level l (h+1..L): D[i][C][t], i < 2^l, C < 2^(L-l+1)
template <typename C>
__global__ void kS_L(const Geo G, int l, C* D)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = G.r;
    const int cb = G.L - l + 1;
    if (e >= (2 * G.N) * r) return;
    int t = (int)(e % r);
    int64_t q = e / r;
    int64_t i = q >> cb, Cc = q & ((1LL << cb) - 1);
    double g = gp(xc(l, i), xw(l), G, t);
    double d = phi(G, g, wc(G.N, cb, Cc)) - phi(G, g, wc(G.N, cb - 1, Cc / 2));
    store(D + e, e2pi(d));
}

// switch at level h with the last H diagonal (right) and first G diagonal (left)
template <typename C>
__global__ void kS_M(const Geo G, int h, C* M)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = G.r;
    if (e >= G.N * r * r) return;
    int s = (int)(e % r);
    int t = (int)((e / r) % r);
    int64_t p = e / (r * r);
    int64_t i = p >> (G.L - h), j = p & ((1LL << (G.L - h)) - 1);
    double cA = xc(h, i), wA = xw(h), cB = wc(G.N, G.L - h, j), wB = ww(G.N, G.L - h);
    double gA = gp(cA, wA, G, t), gB = gp(cB, wB, G, s);
    double d = phi(G, gA, gB) - phi(G, cA, gB) - phi(G, gA, cB);
    store(M + e, e2pi(d));
}

template <typename C>
__global__ void kS_U(const Geo G, const double* x, const int32_t* leaf, int64_t nx, C* U)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nx * G.r) return;
    int t = (int)(e % G.r);
    int64_t n = e / G.r;
    double xn = x[n];
    double cA = xc(G.L, leaf[n]), wA = xw(G.L);
    store(U + e, cscale(lag(G, t, (xn - cA) / wA), e2pi(phi(G, xn, wc(G.N, 0, 0)))));
}

// ---------------------------------------------------------------------------
static Geo make_geo(const ibf_plan* p)
{
    Geo G;
    G.N = p->N;
    G.L = p->L;
    G.r = p->r;
    G.phase = p->phase_id;
    G.nco = (int)p->coef.size() / 2;
    for (int m = 0; m < kMaxCoef; ++m) {
        G.ca[m] = m < G.nco ? p->coef[m] : 0.0;
        G.cb[m] = m < G.nco ? p->coef[G.nco + m] : 0.0;
    }
    for (int t = 0; t < kMaxR; ++t) G.z[t] = t < p->r ? p->z[t] : 0.0;
    return G;
}

static int dalloc(ibf_plan* p, void** ptr, size_t bytes, bool factor)
{
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_error(IBF_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                          cudaGetErrorString(e));
    }
    p->allocations.push_back(*ptr);
    if (factor) p->factor_bytes += bytes;
    return IBF_OK;
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

static void* opt_alloc(ibf_plan* p, size_t bytes)
{
    void* q = nullptr;
    return dalloc(p, &q, bytes, true) ? nullptr : q;
}

static void opt_release(ibf_plan* p, void* q)
{
    auto it = std::find(p->allocations.begin(), p->allocations.end(), q);
    if (it == p->allocations.end()) return;
    cudaFree(q);
    p->allocations.erase(it);
}

int build_explicit(ibf_plan* p)
{
    const Geo G = make_geo(p);
    const int64_t N = p->N;
    const int r = p->r;
    const size_t c16 = sizeof(double2);
    int rc;
    if ((rc = dalloc(p, &p->eV, c16 * N * r, true))) return rc;
    if ((rc = dalloc(p, &p->eM, c16 * N * r * r, true))) return rc;
    if ((rc = dalloc(p, &p->eU, c16 * p->nx * r, true))) return rc;
    p->eblk.assign(p->L + 1, nullptr);
    for (int l = 1; l <= p->L; ++l)
        if ((rc = dalloc(p, &p->eblk[l], c16 * N * 2 * r * r, true))) return rc;
    const int B = 256;
    kE_V<<<nblk(N * r, B), B>>>(G, (double2*)p->eV);
    for (int l = 1; l <= p->L; ++l) kE_blk<<<nblk(N * 2 * r * r, B), B>>>(G, l, p->h, (double2*)p->eblk[l]);
    kE_M<<<nblk(N * r * r, B), B>>>(G, p->h, (double2*)p->eM);
    kE_U<<<nblk(p->nx * r, B), B>>>(G, p->d_x, p->d_leaf, p->nx, (double2*)p->eU);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "explicit construction launch");
    p->nnz = N * r + (int64_t)p->L * N * 2 * r * r + N * r * r + p->nx * r;
    return IBF_OK;
}

template <typename C>
static int build_structured_t(ibf_plan* p)
{
    const Geo G = make_geo(p);
    const int64_t N = p->N;
    const int r = p->r;
    const size_t cs = sizeof(C);
    int rc;
    if ((rc = dalloc(p, &p->sV, cs * N * r, true))) return rc;
    if ((rc = dalloc(p, &p->sM, cs * N * r * r, true))) return rc;
    if ((rc = dalloc(p, &p->sU, cs * p->nx * r, true))) return rc;
    p->stab.assign(p->L + 1, nullptr);
    for (int l = 1; l <= p->L; ++l)
        if ((rc = dalloc(p, &p->stab[l], cs * 2 * N * r, true))) return rc;
    const int B = 256;
    kS_V<C><<<nblk(N * r, B), B>>>(G, (C*)p->sV);
    for (int l = 1; l <= p->h; ++l) kS_Q<C><<<nblk(2 * N * r, B), B>>>(G, l, (C*)p->stab[l]);
    for (int l = p->h + 1; l <= p->L; ++l) kS_L<C><<<nblk(2 * N * r, B), B>>>(G, l, (C*)p->stab[l]);
    kS_M<C><<<nblk(N * r * r, B), B>>>(G, p->h, (C*)p->sM);
    kS_U<C><<<nblk(p->nx * r, B), B>>>(G, p->d_x, p->d_leaf, p->nx, (C*)p->sU);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "structured construction launch");
    p->nnz = N * r + (int64_t)p->L * N * 2 * r * r + N * r * r + p->nx * r;
    return IBF_OK;
}

int build_structured(ibf_plan* p)
{
    return p->dtype == IBF_C128 ? build_structured_t<double2>(p) : build_structured_t<float2>(p);
}

// Chebyshev grid and the universal transfer matrices (host, FP64)
static void host_grid(ibf_plan* p)
{
    const int r = p->r;
    for (int t = 0; t < r; ++t) p->z[t] = 0.5 * std::cos(t * M_PI / (r - 1));
    auto M = [&](int t, double u) {
        double v = 1.0;
        for (int m = 0; m < r; ++m)
            if (m != t) v *= (u - p->z[m]) / (p->z[t] - p->z[m]);
        return v;
    };
    for (int c = 0; c < 2; ++c)
        for (int t = 0; t < r; ++t)
            for (int s = 0; s < r; ++s) p->T[c][t][s] = M(t, (2 * c - 1) / 4.0 + p->z[s] / 2.0);
}

// Profiling: an event is recorded on the apply's stream when the call starts
// and after every kernel; kernel n's duration is the time between the event
// before it and the event after it.
void prof_start(ibf_plan* p, cudaStream_t s)
{
    if (!p->prof_cap || p->prof_n >= p->prof_cap || p->prof_nev >= (int)p->prof_ev.size()) {
        p->prof_last = -1;
        return;
    }
    cudaEventRecord(p->prof_ev[p->prof_nev], s);
    p->prof_last = p->prof_nev++;
}

void prof_mark(ibf_plan* p, cudaStream_t s, int kind)
{
    if (!p->prof_cap || p->prof_last < 0 || p->prof_n >= p->prof_cap || p->prof_nev >= (int)p->prof_ev.size())
        return;
    cudaEventRecord(p->prof_ev[p->prof_nev], s);
    p->prof_a[p->prof_n] = p->prof_last;
    p->prof_b[p->prof_n] = p->prof_nev;
    p->prof_kind[p->prof_n] = kind;
    p->prof_last = p->prof_nev++;
    p->prof_n++;
}

static void free_plan(ibf_plan* p)
{
    if (!p) return;
    delete (Plan2D*)p->p2d;
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : p->hst_ev)
        if (e) cudaEventDestroy(e);
    if (p->hst_in) cudaStreamDestroy(p->hst_in);
    if (p->hst_out) cudaStreamDestroy(p->hst_out);
    for (void* a : p->allocations) cudaFree(a);
    delete p;
}

}  // namespace ibf

using namespace ibf;

extern "C" int ibf_get_last_error(char* buf, size_t len)
{
    if (buf && len) snprintf(buf, len, "%s", g_last_msg);
    return g_last_code;
}

extern "C" int ibf_plan_create(int phase_id, int d, int64_t N, int r, int dtype, ibf_plan** out)
{
    return ibf_plan_create_ex(phase_id, d, N, r, dtype, nullptr, nullptr, out);
}

// 2D multiscale plan (Sec. 5.2); see include/ibf.h
static int create_2d(int phase_id, int64_t N, int r, int dtype, const double* x, const ibf_options* opt,
                     ibf_plan** out)
{
    if (phase_id != IBF_PHASE_FIO2D && phase_id != IBF_PHASE_NUFFT && phase_id != IBF_PHASE_SEPARABLE &&
        phase_id != IBF_PHASE_FIO2D_SERIES)
        return set_error(IBF_ERR_INVALID, "unknown 2D phase id " + std::to_string(phase_id));
    std::vector<double> coef;
    if (phase_id == IBF_PHASE_FIO2D_SERIES) {
        if (!opt || !opt->phase_coef || opt->phase_ncoef < 1 || opt->phase_ncoef > kMaxCoef)
            return set_error(IBF_ERR_INVALID, "IBF_PHASE_FIO2D_SERIES needs phase_coef and 1 <= phase_ncoef <= 16");
        coef.assign(opt->phase_coef, opt->phase_coef + 6 * opt->phase_ncoef);
        for (double v : coef)
            if (!std::isfinite(v)) return set_error(IBF_ERR_INVALID, "phase_coef must be finite");
        // c_d >= (constant terms) - (sum of the other terms' |al| + |be|) must be > 0
        for (int d = 0; d < 2; ++d) {
            double c0 = 0.0, rest = 0.0;
            for (int t = 0; t < opt->phase_ncoef; ++t) {
                const double* row = &coef[6 * t];
                if (row[0] == 0.0 && row[1] == 0.0)
                    c0 += row[2 + 2 * d];
                else
                    rest += std::fabs(row[2 + 2 * d]) + std::fabs(row[3 + 2 * d]);
            }
            if (!(c0 > rest))
                return set_error(IBF_ERR_INVALID, "IBF_PHASE_FIO2D_SERIES: c" + std::to_string(d + 1) +
                                                      " is not bounded away from zero by its terms");
        }
    }
    int n = 1;
    while ((int64_t)n * n < N && n < (1 << 12)) n *= 2;
    if ((int64_t)n * n != N || n < 32 || n > 2048)
        return set_error(IBF_ERR_INVALID, "2D: N must be n^2 with n a power of two in [32, 2048]");
    if (r != 5 && r != 7 && r != 9) return set_error(IBF_ERR_UNSUPPORTED, "2D: r must be 5, 7 or 9");
    if (dtype != IBF_C128 && dtype != IBF_C64_FP32) return set_error(IBF_ERR_UNSUPPORTED, "2D: dtype");
    if (x) return set_error(IBF_ERR_UNSUPPORTED, "2D: only the uniform grid X is supported");
    ibf_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.form == IBF_FORM_EXPLICIT || o.form == IBF_FORM_OPTIMAL || o.form == IBF_FORM_OPTIMAL_IN)
        return set_error(IBF_ERR_UNSUPPORTED, "2D: structured form only");
    ibf_plan* p = new ibf_plan();
    p->phase_id = phase_id;
    p->coef = coef;
    p->d = 2;
    p->r = r;
    p->dtype = dtype;
    p->form = IBF_FORM_STRUCTURED;
    p->N = N;
    p->nx = N;
    p->L = 0;
    while ((1 << p->L) < n) ++p->L;
    p->h = (p->L + 1) / 2;
    p->max_nrhs = o.max_nrhs > 0 ? o.max_nrhs : 32;
    host_grid(p);
    Plan2D* P = new Plan2D();
    P->n = n;
    P->center = 16;
    p->p2d = P;
    int rc = build_2d(p);
    if (rc) {
        free_plan(p);
        return rc;
    }
    const size_t esz = dtype == IBF_C128 ? sizeof(double2) : sizeof(float2);
    for (int b = 0; b < 2; ++b)
        if ((rc = dalloc(p, &P->ws[b], esz * P->ws_elems, false))) {
            free_plan(p);
            return rc;
        }
    p->ws_bytes = 2 * esz * P->ws_elems;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_error(e, "2D plan construction");
    }
    *out = p;
    return IBF_OK;
}

extern "C" int ibf_plan_create_ex(int phase_id, int d, int64_t N, int r, int dtype, const double* x,
                                  const ibf_options* opt, ibf_plan** out)
{
    if (!out) return set_error(IBF_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (d == 2) return create_2d(phase_id, N, r, dtype, x, opt, out);
    if (d != 1) return set_error(IBF_ERR_INVALID, "d must be 1 or 2");
    if (phase_id != IBF_PHASE_NUFFT && phase_id != IBF_PHASE_FIO1D && phase_id != IBF_PHASE_SEPARABLE &&
        phase_id != IBF_PHASE_FIO1D_SERIES)
        return set_error(IBF_ERR_INVALID, "unknown 1D phase id " + std::to_string(phase_id));
    std::vector<double> coef;
    if (phase_id == IBF_PHASE_FIO1D_SERIES) {
        if (!opt || !opt->phase_coef || opt->phase_ncoef < 1 || opt->phase_ncoef > kMaxCoef)
            return set_error(IBF_ERR_INVALID, "IBF_PHASE_FIO1D_SERIES needs phase_coef and 1 <= phase_ncoef <= 16");
        coef.assign(opt->phase_coef, opt->phase_coef + 2 * opt->phase_ncoef);
        for (double v : coef)
            if (!std::isfinite(v)) return set_error(IBF_ERR_INVALID, "phase_coef must be finite");
    }
    if (N < 4 || N > (1LL << 24) || (N & (N - 1)))
        return set_error(IBF_ERR_INVALID, "N must be a power of two in [4, 2^24]");
    if (r < 3 || r > kMaxR) return set_error(IBF_ERR_INVALID, "r must be in [3, 16]");
    if (dtype != IBF_C128 && dtype != IBF_C64_FP32 && dtype != IBF_C64_BF16X3 && dtype != IBF_C64_TF32X3)
        return set_error(IBF_ERR_INVALID, "unknown dtype");
    ibf_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    int form = o.form == IBF_FORM_AUTO ? (dtype == IBF_C128 ? IBF_FORM_EXPLICIT : IBF_FORM_STRUCTURED) : o.form;
    if (form != IBF_FORM_EXPLICIT && form != IBF_FORM_STRUCTURED && form != IBF_FORM_OPTIMAL &&
        form != IBF_FORM_OPTIMAL_IN)
        return set_error(IBF_ERR_INVALID, "unknown form");
    const bool optimal = form == IBF_FORM_OPTIMAL || form == IBF_FORM_OPTIMAL_IN;
    if (optimal) {
        if (dtype != IBF_C128 && dtype != IBF_C64_FP32)
            return set_error(IBF_ERR_UNSUPPORTED, "the optimal form is FP64 or FP32");
        if (r > 12) return set_error(IBF_ERR_UNSUPPORTED, "the optimal form supports r <= 12");
        if (o.rank < 1 || o.rank > r) return set_error(IBF_ERR_INVALID, "optimal form: rank must be in [1, r]");
    }
    if (form == IBF_FORM_EXPLICIT && dtype != IBF_C128 && dtype != IBF_C64_FP32)
        return set_error(IBF_ERR_UNSUPPORTED, "the explicit form is FP64 or FP32");
    if (dtype == IBF_C64_BF16X3)
        return set_error(IBF_ERR_UNSUPPORTED, "split-BF16 tensor-core apply is not built (IBF_C64_TF32X3 is)");
    if (dtype == IBF_C64_TF32X3 && form != IBF_FORM_STRUCTURED)
        return set_error(IBF_ERR_UNSUPPORTED, "IBF_C64_TF32X3 is the structured form only");
    if (form == IBF_FORM_STRUCTURED && !fused_supports_r(r))
        return set_error(IBF_ERR_UNSUPPORTED, "structured form supports r in {5, 7, 9, 11}");

    int L = 0;
    while ((1LL << L) < N) ++L;
    int h = o.h > 0 ? o.h : L / 2;
    if (h < 1 || h > L - 1) return set_error(IBF_ERR_INVALID, "switch level h must be in [1, L-1]");

    // target points: validate, then sort by leaf on the host (plan set-up)
    std::vector<double> xs(N);
    std::vector<int32_t> perm(N), off(N + 1, 0), leaf(N);
    if (x) {
        for (int64_t n = 0; n < N; ++n) {
            if (!(x[n] >= 0.0 && x[n] < 1.0)) return set_error(IBF_ERR_INVALID, "points must lie in [0,1)");
        }
        std::iota(perm.begin(), perm.end(), 0);
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return x[a] < x[b]; });
        for (int64_t n = 0; n < N; ++n) xs[n] = x[perm[n]];
    } else {
        for (int64_t n = 0; n < N; ++n) {
            xs[n] = (double)n / (double)N;
            perm[n] = (int32_t)n;
        }
    }
    for (int64_t n = 0; n < N; ++n) {
        int64_t i = (int64_t)std::floor(xs[n] * (double)N);
        i = std::min<int64_t>(std::max<int64_t>(i, 0), N - 1);
        leaf[n] = (int32_t)i;
        off[i + 1]++;
    }
    for (int64_t i = 0; i < N; ++i) off[i + 1] += off[i];

    ibf_plan* p = new ibf_plan();
    p->phase_id = phase_id;
    p->coef = coef;
    p->d = d;
    p->r = r;
    p->dtype = dtype;
    p->form = form;
    p->L = L;
    p->h = h;
    p->N = N;
    p->nx = N;
    p->max_nrhs = o.max_nrhs > 0 ? o.max_nrhs : (form == IBF_FORM_STRUCTURED ? 64 : 8);
    p->kfuse = o.levels_per_launch;
    p->rtile = o.rhs_tile;
    p->user_kfuse = o.levels_per_launch > 0;
    p->user_rtile = o.rhs_tile > 0;
    if (p->user_kfuse && p->kfuse > kMaxFuse) { free_plan(p); return set_error(IBF_ERR_INVALID, "levels_per_launch > 10"); }
    if (p->user_rtile && (p->rtile > 64 || (p->rtile & (p->rtile - 1)))) {
        free_plan(p);
        return set_error(IBF_ERR_INVALID, "rhs_tile must be a power of two <= 64");
    }
    host_grid(p);

    int rc;
    if ((rc = dalloc(p, (void**)&p->d_x, sizeof(double) * N, false)) ||
        (rc = dalloc(p, (void**)&p->d_perm, sizeof(int32_t) * N, false)) ||
        (rc = dalloc(p, (void**)&p->d_off, sizeof(int32_t) * (N + 1), false)) ||
        (rc = dalloc(p, (void**)&p->d_leaf, sizeof(int32_t) * N, false))) {
        free_plan(p);
        return rc;
    }
    cudaMemcpy(p->d_x, xs.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_perm, perm.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_off, off.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_leaf, leaf.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);

    rc = form == IBF_FORM_STRUCTURED ? build_structured(p) : build_explicit(p);
    if (!rc && optimal) {
        rc = compress_optimal(p, o.rank, opt_alloc, opt_release);
        if (!rc && form == IBF_FORM_OPTIMAL_IN) rc = sweep_in_optimal(p, off, opt_alloc, opt_release);
        if (!rc) p->factor_bytes = sizeof(double2) * (size_t)p->nnz;
    }
    // FP32 explicit and optimal plans: built in FP64, stored and applied in FP32
    if (!rc && form != IBF_FORM_STRUCTURED && dtype == IBF_C64_FP32) rc = explicit_demote(p, opt_alloc, opt_release);
    if (rc) {
        free_plan(p);
        return rc;
    }
    // apply workspace: two Lambda buffers of N r max_nrhs complex
    size_t esz = dtype == IBF_C128 ? sizeof(double2) : sizeof(float2);
    size_t wsb = esz * (size_t)N * r * p->max_nrhs;
    for (int b = 0; b < 2; ++b)
        if ((rc = dalloc(p, &p->ws[b], wsb, false))) {
            free_plan(p);
            return rc;
        }
    p->ws_bytes = 2 * wsb;
    if (dtype == IBF_C64_TF32X3 || (dtype == IBF_C64_FP32 && form != IBF_FORM_STRUCTURED)) {
        // status word of the bounded device-side waits (ibf_plan_status)
        if ((rc = dalloc(p, (void**)&p->d_status, sizeof(int), false))) {
            free_plan(p);
            return rc;
        }
        cudaMemset(p->d_status, 0, sizeof(int));
    }
    if (form == IBF_FORM_STRUCTURED) {
        fused_choose_shape(p);
        // commit the static-scratch array on this device now, while the
        // caller may still allocate; a failure here is reported again by
        // ibf_apply_static_scratch, the only user of the array
        if (static_scratch_prepare(p) != IBF_OK) cudaGetLastError();
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_error(e, "plan construction");
    }
    *out = p;
    return IBF_OK;
}

extern "C" int ibf_plan_destroy(ibf_plan* p)
{
    if (!p) return IBF_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    return IBF_OK;
}

static int check_apply(ibf_plan* p, const void* a, void* b, int nrhs)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    if (!a || !b) return set_error(IBF_ERR_INVALID, "NULL vector pointer");
    if (nrhs < 1) return set_error(IBF_ERR_INVALID, "nrhs must be >= 1");
    size_t al = p->dtype == IBF_C128 ? 16 : 8;
    if (((uintptr_t)a % al) || ((uintptr_t)b % al)) return set_error(IBF_ERR_INVALID, "misaligned vector pointer");
    size_t bytes = al * (size_t)p->N * nrhs;
    const char* ca = (const char*)a;
    const char* cb = (const char*)b;
    if (ca < cb + bytes && cb < ca + bytes) return set_error(IBF_ERR_INVALID, "input and output overlap");
    return IBF_OK;
}

extern "C" int ibf_apply(ibf_plan* p, const void* g, void* u, int nrhs, ibf_stream_t stream)
{
    int rc = check_apply(p, g, u, nrhs);
    if (rc) return rc;
    if (p->d == 2) return plan_note(p, apply_2d(p, g, u, nrhs, (cudaStream_t)stream));
    if (p->form != IBF_FORM_STRUCTURED) return plan_note(p, explicit_apply(p, g, u, nrhs, (cudaStream_t)stream));
    return plan_note(p, fused_apply(p, g, u, nrhs, false, (cudaStream_t)stream));
}

extern "C" int ibf_apply_adjoint(ibf_plan* p, const void* y, void* g, int nrhs, ibf_stream_t stream)
{
    int rc = check_apply(p, y, g, nrhs);
    if (rc) return rc;
    if (p->d == 2) return plan_note(p, apply_2d_adjoint(p, y, g, nrhs, (cudaStream_t)stream));
    if (p->form != IBF_FORM_STRUCTURED) return plan_note(p, explicit_adjoint(p, y, g, nrhs, (cudaStream_t)stream));
    return plan_note(p, fused_apply(p, y, g, nrhs, true, (cudaStream_t)stream));
}

extern "C" int ibf_plan_status(ibf_plan* p)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    if (p->d_status) {
        // plans whose kernels wait on mbarriers: a bounded wait that expired
        int dev = 0;
        if (cudaMemcpy(&dev, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return set_error(IBF_ERR_CUDA, "plan status: reading the device status word failed");
        if (dev) {
            cudaMemset(p->d_status, 0, sizeof(int));
            plan_note(p, IBF_ERR_TIMEOUT);
        }
    }
    const int st = p->sticky;
    p->sticky = IBF_OK;
    if (st != IBF_OK) return set_error(st, "sticky status of the plan: an earlier apply failed or its batch timed out");
    return IBF_OK;
}

// Host-buffer apply: chunks of `hst_chunk` columns go through two device
// staging slots.  Chunk j (slot s = j % 2): copy-in stream waits until the
// apply of chunk j-2 has read slot s, copies the chunk in; `stream` waits for
// that copy and for the copy-out of chunk j-2 from slot s, applies; copy-out
// stream waits for the apply and copies the result out.  So the copies of
// neighbouring chunks overlap the apply of the current one.
static int host_setup(ibf_plan* p)
{
    if (p->hst_buf) return IBF_OK;
    const size_t esz = p->dtype == IBF_C128 ? 16 : 8;
    const int tile = (p->d == 1 && p->form == IBF_FORM_STRUCTURED && p->rtile > 0) ? p->rtile : 16;
    p->hst_chunk = std::max(1, std::min(p->max_nrhs, tile));
    cudaError_t e;
    for (cudaEvent_t& ev : p->hst_ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_error(e, "host apply: cudaEventCreate");
    if ((e = cudaStreamCreateWithFlags(&p->hst_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&p->hst_out, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_error(e, "host apply: cudaStreamCreate");
    void* buf = nullptr;
    if ((e = cudaMalloc(&buf, 4 * esz * (size_t)p->N * p->hst_chunk)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(IBF_ERR_OOM, "host apply: staging buffers");
    }
    p->allocations.push_back(buf);
    p->hst_buf = buf;
    return IBF_OK;
}

extern "C" int ibf_apply_host(ibf_plan* p, const void* hin, void* hout, int nrhs, int flags, ibf_stream_t stream)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    if (!hin || !hout) return set_error(IBF_ERR_INVALID, "NULL vector pointer");
    if (nrhs < 1) return set_error(IBF_ERR_INVALID, "nrhs must be >= 1");
    if (flags & ~(IBF_HOST_ADJOINT | IBF_HOST_PIPELINE | IBF_HOST_DEFER))
        return set_error(IBF_ERR_INVALID, "unknown flag bits");
    const bool adjoint = flags & IBF_HOST_ADJOINT;
    const size_t esz = p->dtype == IBF_C128 ? 16 : 8;
    if (((uintptr_t)hin % esz) || ((uintptr_t)hout % esz)) return set_error(IBF_ERR_INVALID, "misaligned vector pointer");
    int rc = host_setup(p);
    if (rc) return plan_note(p, rc);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t col = esz * (size_t)p->N;
    const int ch = p->hst_chunk;
    char* slot_in[2] = {(char*)p->hst_buf, (char*)p->hst_buf + col * ch};
    char* slot_out[2] = {(char*)p->hst_buf + 2 * col * ch, (char*)p->hst_buf + 3 * col * ch};
    cudaEvent_t ev0 = p->hst_ev[0], *h2d = p->hst_ev + 1, *app = p->hst_ev + 3, *d2h = p->hst_ev + 5;
    cudaError_t e;
    const size_t total = col * (size_t)nrhs;
    const bool first = p->hst_prev_out == nullptr;
    const bool pipelined = (flags & IBF_HOST_PIPELINE) && !first;
    if (pipelined) {
        // the copy-in into slot s waits only for the previous call's last
        // apply that read slot s (in the loop below), so the first chunk's
        // copy-in runs under the previous call's last apply; if that call's
        // output overlaps this input, it waits for its copy-outs too
        const char* po = (const char*)p->hst_prev_out;
        const char* ci = (const char*)hin;
        if (ci < po + p->hst_prev_bytes && po < ci + total) {
            cudaStreamWaitEvent(p->hst_in, d2h[0], 0);
            cudaStreamWaitEvent(p->hst_in, d2h[1], 0);
        }
    } else {
        // earlier work on `stream` (a previous call's applies) comes first
        if ((e = cudaEventRecord(ev0, st)) != cudaSuccess) return cuda_error(e, "host apply: event");
        cudaStreamWaitEvent(p->hst_in, ev0, 0);
        cudaStreamWaitEvent(p->hst_out, ev0, 0);
    }
    p->hst_prev_out = hout;
    p->hst_prev_bytes = total;
    // copy-outs of an earlier deferred call may still read the staging slots
    // this call's first applies write
    const bool after_deferred = p->hst_deferred;
    const int nch = (nrhs + ch - 1) / ch;
    for (int j = 0; j < nch; ++j) {
        const int s = j & 1, c0 = j * ch, nc = std::min(ch, nrhs - c0);
        if (j >= 2 || pipelined) cudaStreamWaitEvent(p->hst_in, app[s], 0);
        if ((e = cudaMemcpyAsync(slot_in[s], (const char*)hin + col * c0, col * nc, cudaMemcpyHostToDevice,
                                 p->hst_in)) != cudaSuccess)
            return plan_note(p, cuda_error(e, "host apply: copy in"));
        cudaEventRecord(h2d[s], p->hst_in);
        cudaStreamWaitEvent(st, h2d[s], 0);
        if (j >= 2 || after_deferred) cudaStreamWaitEvent(st, d2h[s], 0);
        rc = adjoint ? ibf_apply_adjoint(p, slot_in[s], slot_out[s], nc, stream)
                     : ibf_apply(p, slot_in[s], slot_out[s], nc, stream);
        if (rc) return rc;
        cudaEventRecord(app[s], st);
        cudaStreamWaitEvent(p->hst_out, app[s], 0);
        if ((e = cudaMemcpyAsync((char*)hout + col * c0, slot_out[s], col * nc, cudaMemcpyDeviceToHost,
                                 p->hst_out)) != cudaSuccess)
            return plan_note(p, cuda_error(e, "host apply: copy out"));
        cudaEventRecord(d2h[s], p->hst_out);
    }
    if (flags & IBF_HOST_DEFER) {
        // the copy-outs stay on the copy stream: the next call or
        // ibf_host_flush orders `stream` after them
        p->hst_deferred = true;
    } else {
        // `stream` completes only after every copy-out, earlier deferred ones
        // included (both slots' latest copy-outs)
        cudaStreamWaitEvent(st, d2h[0], 0);
        cudaStreamWaitEvent(st, d2h[1], 0);
        p->hst_deferred = false;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : plan_note(p, cuda_error(e, "host apply"));
}

extern "C" int ibf_host_flush(ibf_plan* p, ibf_stream_t stream)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    if (!p->hst_buf || !p->hst_deferred) return IBF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamWaitEvent(st, p->hst_ev[5], 0);   // d2h of slot 0
    cudaStreamWaitEvent(st, p->hst_ev[6], 0);   // d2h of slot 1
    p->hst_deferred = false;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IBF_OK : plan_note(p, cuda_error(e, "host flush"));
}

extern "C" int ibf_plan_profile_begin(ibf_plan* p, int cap)
{
    if (!p || cap < 1 || cap > (1 << 20)) return set_error(IBF_ERR_INVALID, "bad plan or cap");
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.assign(2 * cap, nullptr);
    for (auto& e : p->prof_ev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return cuda_error(err, "cudaEventCreate");
    }
    p->prof_a.assign(cap, 0);
    p->prof_b.assign(cap, 0);
    p->prof_kind.assign(cap, -1);
    p->prof_n = 0;
    p->prof_nev = 0;
    p->prof_last = -1;
    p->prof_cap = cap;
    return IBF_OK;
}

extern "C" int ibf_plan_profile_end(ibf_plan* p, float* ms, int* kind, int cap_out, int* count)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    int n = p->prof_n;
    int rc = IBF_OK;
    for (int e = 0; e < n; ++e) {
        float t = 0.f;
        cudaError_t err = cudaEventSynchronize(p->prof_ev[p->prof_b[e]]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, p->prof_ev[p->prof_a[e]], p->prof_ev[p->prof_b[e]]);
        if (err != cudaSuccess) {
            rc = cuda_error(err, "profile events");
            break;
        }
        if (e < cap_out) {
            if (ms) ms[e] = t;
            if (kind) kind[e] = p->prof_kind[e];
        }
    }
    if (count) *count = n;
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    p->prof_cap = 0;
    p->prof_n = 0;
    p->prof_nev = 0;
    p->prof_last = -1;
    return rc;
}

extern "C" int ibf_plan_query(const ibf_plan* p, int what, int64_t* v)
{
    if (!p || !v) return set_error(IBF_ERR_INVALID, "NULL argument");
    switch (what) {
    case IBF_Q_N: *v = p->N; break;
    case IBF_Q_L: *v = p->L; break;
    case IBF_Q_H: *v = p->h; break;
    case IBF_Q_R: *v = p->r; break;
    case IBF_Q_DTYPE: *v = p->dtype; break;
    case IBF_Q_FORM: *v = p->form; break;
    case IBF_Q_FACTOR_BYTES: *v = (int64_t)p->factor_bytes; break;
    case IBF_Q_WORKSPACE_BYTES: *v = (int64_t)p->ws_bytes; break;
    case IBF_Q_MAX_NRHS: *v = p->max_nrhs; break;
    case IBF_Q_NNZ: *v = p->nnz; break;
    case IBF_Q_LAUNCHES:
        *v = p->d == 2 ? launches_2d(p) : (p->form != IBF_FORM_STRUCTURED ? explicit_launches(p) : fused_launches(p));
        break;
    case IBF_Q_LEVELS_PER_LAUNCH: *v = p->kfuse; break;
    case IBF_Q_RHS_TILE: *v = p->rtile; break;
    case IBF_Q_RANK: *v = p->ra > 0 ? p->ra : p->r; break;
    default: return set_error(IBF_ERR_INVALID, "unknown query");
    }
    return IBF_OK;
}
