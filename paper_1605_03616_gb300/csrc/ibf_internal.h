// Internal declarations shared by the translation units of the IBF library.
// The public C ABI is include/ibf.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ibf.h"

namespace ibf {

constexpr int kMaxR = 16;       // Chebyshev points per box
constexpr int kMaxFuse = 10;    // butterfly levels fused in one structured kernel
constexpr int kMaxCoef = 16;    // terms of the coefficient series of the series phases

// Host-side record of the last error of the calling thread.
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);

}  // namespace ibf

struct ibf_plan {
    int phase_id = 0, d = 1, r = 0, dtype = 0, form = 0;
    std::vector<double> coef;   // series phases: a_0..a_{M-1}, b_0..b_{M-1} (1D) or M rows of 6 (2D)
    int L = 0, h = 0;
    int64_t N = 0, nx = 0;
    int max_nrhs = 0;
    int kfuse = 0, rtile = 0;   // structured form launch shape
    int ra = 0;                 // optimal form: rank r0 of the compressed blocks (0: r)
    // optimal form after the sweep-in stage: rank of Lambda^l before the
    // switch (rk_h[l], l = 0..h) and after it (rk_g[l], l = h..L); empty:
    // every level has rank ra (or r)
    std::vector<int> rk_h, rk_g;
    bool user_kfuse = false, user_rtile = false;
    // sticky status (ibf_plan_status): the first error of an apply on this
    // plan after its arguments were accepted, or IBF_ERR_TIMEOUT from a
    // persistent batch holding the plan; read and cleared by ibf_plan_status
    mutable int sticky = 0;
    int* d_status = nullptr;   // device word set when a bounded wait expires (tensor-core levels of
                               // IBF_C64_TF32X3, bulk-copy levels of complex64 explicit forms)

    // Chebyshev grid on [-1/2,1/2] and the two child-to-parent Lagrange
    // transfer matrices T_c[t][s] = M_t((2c-1)/4 + z_s/2)   (Sec. 2.1)
    double z[ibf::kMaxR];
    double T[2][ibf::kMaxR][ibf::kMaxR];

    // target points, sorted by leaf; perm[n] = caller index of sorted point n;
    // off[i]..off[i+1] = sorted points in leaf i (N+1 entries)
    double* d_x = nullptr;
    int32_t* d_perm = nullptr;
    int32_t* d_off = nullptr;
    int32_t* d_leaf = nullptr;

    // explicit form (complex128): V[k][t], blk[l][p][c][t][s], M[p][t][s], U[n][t]
    void* eV = nullptr;
    void* eM = nullptr;
    void* eU = nullptr;
    std::vector<void*> eblk;   // index 1..L

    // structured form (complex of the apply precision):
    //   sV[k][t]         = M_t((xi_k - c_B)/w_B) e(Phi(c_root, xi_k))
    //   stab[l][i][C][s] = e(Phi(c_{A^l_i}, g_s) - Phi(c_{A^{l-1}_{i/2}}, g_s)),  l <= h
    //   stab[l][i][C][t] = e(Phi(g^{A^l_i}_t, c_C) - Phi(g^{A^l_i}_t, c_{parent(C)})), l > h
    //   sM[p][t][s]      = the switch block with both neighbouring diagonals merged
    //   sU[n][t]         = e(Phi(x_n, 0)) M_t((x_n - c_A)/w_A)
    void* sV = nullptr;
    void* sM = nullptr;
    void* sU = nullptr;
    std::vector<void*> stab;   // index 1..L

    // 2D multiscale plan (struct Plan2D, ibf_2d.h), d = 2 only
    void* p2d = nullptr;

    void* ws[2] = {nullptr, nullptr};   // apply workspace (ping-pong Lambda buffers)

    // host-buffer apply (ibf_apply_host), set up by its first call: device
    // staging slots [2][in|out][N x chunk], two copy streams and their events
    void* hst_buf = nullptr;
    int hst_chunk = 0;
    cudaStream_t hst_in = nullptr, hst_out = nullptr;
    cudaEvent_t hst_ev[7] = {};   // start, h2d[2], apply[2], d2h[2]
    const void* hst_prev_out = nullptr;   // out_host of the previous call (IBF_HOST_PIPELINE)
    size_t hst_prev_bytes = 0;
    bool hst_deferred = false;            // copy-outs not yet ordered before `stream` (IBF_HOST_DEFER)
    size_t factor_bytes = 0, ws_bytes = 0;
    int64_t nnz = 0;
    std::vector<void*> allocations;

    // optional per-launch timing (ibf_plan_profile_begin/end): kernel n ran
    // between events prof_a[n] and prof_b[n]
    int prof_cap = 0, prof_n = 0, prof_nev = 0, prof_last = -1;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_a, prof_b, prof_kind;
};

namespace ibf {

// per-launch timing helpers (no-ops unless profiling is on)
void prof_start(ibf_plan* p, cudaStream_t s);
void prof_mark(ibf_plan* p, cudaStream_t s, int kind);

// construction (ibf_plan.cu)
int build_explicit(ibf_plan* p);
int build_structured(ibf_plan* p);

// optimal form (ibf_optimal.cu): compress the explicit factors to rank r0;
// alloc returns device memory owned by the plan (nullptr on failure), release
// frees one such block
int compress_optimal(ibf_plan* p, int r0, void* (*alloc)(ibf_plan*, size_t), void (*release)(ibf_plan*, void*));
int explicit_demote(ibf_plan* p, void* (*alloc)(ibf_plan*, size_t), void (*release)(ibf_plan*, void*));
int sweep_in_optimal(ibf_plan* p, const std::vector<int32_t>& off, void* (*alloc)(ibf_plan*, size_t),
                     void (*release)(ibf_plan*, void*));

// explicit-form apply (ibf_explicit.cu), FP64
int explicit_apply(ibf_plan* p, const void* g, void* u, int nrhs, cudaStream_t s);
int explicit_adjoint(ibf_plan* p, const void* y, void* g, int nrhs, cudaStream_t s);
int explicit_launches(const ibf_plan* p);

// structured-form apply (ibf_fused.cu), FP32 or FP64
int fused_apply(ibf_plan* p, const void* g, void* u, int nrhs, bool adjoint, cudaStream_t s);
int fused_launches(const ibf_plan* p);
bool fused_supports_r(int r);
void fused_choose_shape(ibf_plan* p);

// record a failure of an apply on p in its sticky status; returns rc
inline int plan_note(const ibf_plan* p, int rc)
{
    if (rc != IBF_OK && p && p->sticky == IBF_OK) p->sticky = rc;
    return rc;
}

// static-scratch apply (ibf_static.cu): per-device set-up of its array and
// weights for a new 1D structured plan (see ibf_apply_static_scratch)
int static_scratch_prepare(const ibf_plan* p);

}  // namespace ibf
