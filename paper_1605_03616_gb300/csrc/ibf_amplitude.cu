// ibf_apply_amplitude: kernels K(x, xi) = a(x, xi) e(Phi(x, xi)) with a
// non-unit amplitude (eq. FIO).  The paper sets a = 1 after noting that a
// smooth amplitude is numerically low rank on X x Omega (Sec. 1).  Given that
// low-rank form a(x, xi) = sum_{t<q} alpha_t(x) beta_t(xi), the operator is
//
//   A   = sum_t diag(alpha_t) K diag(beta_t),
//   A^* = sum_t diag(conj beta_t) K^* diag(conj alpha_t),
//
// with K the plan's phase-only operator.  One pass over m amplitude terms:
//   spread : w_in[:, t nrhs + c] = f_t .* in[:, c]        (f = beta, or conj alpha)
//   apply  : w_out = K w_in  (or K^* w_in) on m nrhs columns, any plan form
//   gather : out[:, c] (+)= sum_t f'_t .* w_out[:, t nrhs + c]  (f' = alpha, or conj beta)
// Spread and gather are streaming kernels: each thread owns one row k of one
// column c, reads in[k, c] (or the m products) once and the factor rows from
// L2 (the factor arrays are N q elements, read once per column).
#include <algorithm>
#include <climits>
#include <initializer_list>

#include "ibf_internal.h"

namespace ibf {
namespace {

template <typename T> struct AmpCx;
template <> struct AmpCx<float> { typedef float2 T; };
template <> struct AmpCx<double> { typedef double2 T; };

// a * b, or conj(a) * b
template <bool CONJ, typename cx>
__device__ __forceinline__ cx amp_mul(cx a, cx b)
{
    const auto ay = CONJ ? -a.y : a.y;
    cx o;
    o.x = fma(a.x, b.x, -ay * b.y);
    o.y = fma(a.x, b.y, ay * b.x);
    return o;
}

constexpr int kAmpThreads = 256;

// w[(t nrhs + c) N + k] = f[(t0 + t) N + k] (conj if CONJ) * in[c N + k],
// t < m, c < nrhs, k < N.
template <typename cx, bool CONJ>
__global__ void __launch_bounds__(kAmpThreads) kA_spread(const cx* __restrict__ in, const cx* __restrict__ f,
                                                        cx* __restrict__ w, int64_t N, int nrhs, int t0, int m)
{
    for (int c = blockIdx.y; c < nrhs; c += gridDim.y)
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
            const cx v = in[(int64_t)c * N + k];
            for (int t = 0; t < m; ++t)
                w[((int64_t)t * nrhs + c) * N + k] = amp_mul<CONJ>(f[(int64_t)(t0 + t) * N + k], v);
        }
}

// out[c N + k] (+)= sum_{t<m} f[(t0 + t) N + k] (conj if CONJ) * w[(t nrhs + c) N + k]
template <typename cx, bool CONJ>
__global__ void __launch_bounds__(kAmpThreads) kA_gather(const cx* __restrict__ w, const cx* __restrict__ f,
                                                        cx* __restrict__ out, int64_t N, int nrhs, int t0, int m,
                                                        int accumulate)
{
    for (int c = blockIdx.y; c < nrhs; c += gridDim.y)
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
            cx acc;
            if (accumulate) {
                acc = out[(int64_t)c * N + k];
            } else {
                acc.x = 0;
                acc.y = 0;
            }
            for (int t = 0; t < m; ++t) {
                const cx p = amp_mul<CONJ>(f[(int64_t)(t0 + t) * N + k], w[((int64_t)t * nrhs + c) * N + k]);
                acc.x += p.x;
                acc.y += p.y;
            }
            out[(int64_t)c * N + k] = acc;
        }
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const char* ca = (const char*)a;
    const char* cb = (const char*)b;
    return ca < cb + nb && cb < ca + na;
}

template <typename Real>
int amplitude_t(ibf_plan* p, const void* alpha, const void* beta, int q, const void* in, void* out, int nrhs,
                int adjoint, void* work, int m, cudaStream_t st)
{
    typedef typename AmpCx<Real>::T cx;
    const int64_t N = p->N;
    // blocks: enough to cover N once per column, capped so that a launch
    // stays near 8 resident CTAs of 256 threads per SM on 152 SMs per column
    const int64_t nb = std::min<int64_t>((N + kAmpThreads - 1) / kAmpThreads, 152 * 8);
    cx* w_in = (cx*)work;
    cx* w_out = w_in + (int64_t)m * nrhs * N;
    // forward: in = g scaled by beta, out = u gathered with alpha;
    // adjoint: in = y scaled by conj alpha, out = g gathered with conj beta
    const cx* f_in = (const cx*)(adjoint ? alpha : beta);
    const cx* f_out = (const cx*)(adjoint ? beta : alpha);
    for (int t0 = 0; t0 < q; t0 += m) {
        const int mt = std::min(m, q - t0);
        dim3 grid((unsigned)nb, (unsigned)std::min(nrhs, 65535));
        if (adjoint)
            kA_spread<cx, true><<<grid, kAmpThreads, 0, st>>>((const cx*)in, f_in, w_in, N, nrhs, t0, mt);
        else
            kA_spread<cx, false><<<grid, kAmpThreads, 0, st>>>((const cx*)in, f_in, w_in, N, nrhs, t0, mt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "amplitude: spread kernel");
        const int rc = adjoint ? ibf_apply_adjoint(p, w_in, w_out, mt * nrhs, st)
                               : ibf_apply(p, w_in, w_out, mt * nrhs, st);
        if (rc) return rc;
        const int acc = t0 > 0 ? 1 : 0;
        if (adjoint)
            kA_gather<cx, true><<<grid, kAmpThreads, 0, st>>>(w_out, f_out, (cx*)out, N, nrhs, t0, mt, acc);
        else
            kA_gather<cx, false><<<grid, kAmpThreads, 0, st>>>(w_out, f_out, (cx*)out, N, nrhs, t0, mt, acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "amplitude: gather kernel");
    }
    return IBF_OK;
}

}  // namespace
}  // namespace ibf

using namespace ibf;

extern "C" int ibf_apply_amplitude(ibf_plan* p, const void* alpha, const void* beta, int q, const void* in,
                                   void* out, int nrhs, int adjoint, void* work, int64_t work_elems,
                                   ibf_stream_t stream)
{
    if (!p) return set_error(IBF_ERR_INVALID, "plan is NULL");
    if (!alpha || !beta || !in || !out || !work) return set_error(IBF_ERR_INVALID, "NULL pointer");
    if (q < 1) return set_error(IBF_ERR_INVALID, "q (amplitude terms) must be >= 1");
    if (nrhs < 1) return set_error(IBF_ERR_INVALID, "nrhs must be >= 1");
    const size_t esz = p->dtype == IBF_C128 ? 16 : 8;
    for (const void* a : {(const void*)alpha, (const void*)beta, in, (const void*)out, (const void*)work})
        if ((uintptr_t)a % esz) return set_error(IBF_ERR_INVALID, "misaligned pointer");
    const int64_t N = p->N;
    const int64_t col_pair = 2 * N * (int64_t)nrhs;         // elements of one term's two scratch columns
    if (work_elems < col_pair) return set_error(IBF_ERR_INVALID, "work holds fewer than 2 N nrhs elements");
    const int64_t m64 = std::min<int64_t>(q, work_elems / col_pair);
    if (m64 * nrhs > INT_MAX) return set_error(IBF_ERR_INVALID, "q nrhs exceeds the column count of one apply");
    const int m = (int)m64;
    const size_t vb = esz * (size_t)N * nrhs;                 // bytes of in / out
    const size_t fb = esz * (size_t)N * q;                    // bytes of alpha / beta
    const size_t wb = esz * (size_t)(2 * m64 * N * nrhs);     // bytes of work used
    if (overlaps(in, vb, out, vb)) return set_error(IBF_ERR_INVALID, "input and output overlap");
    if (overlaps(out, vb, alpha, fb) || overlaps(out, vb, beta, fb))
        return set_error(IBF_ERR_INVALID, "output overlaps an amplitude factor");
    if (overlaps(work, wb, in, vb) || overlaps(work, wb, out, vb) || overlaps(work, wb, alpha, fb) ||
        overlaps(work, wb, beta, fb))
        return set_error(IBF_ERR_INVALID, "work overlaps another argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->dtype == IBF_C128)
        return plan_note(p, amplitude_t<double>(p, alpha, beta, q, in, out, nrhs, adjoint, work, m, st));
    return plan_note(p, amplitude_t<float>(p, alpha, beta, q, in, out, nrhs, adjoint, work, m, st));
}
