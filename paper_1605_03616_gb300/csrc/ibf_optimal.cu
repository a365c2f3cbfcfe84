// Optimal IBF, sweep-out stage (Sec. 4.1-4.2) and sweep-in stage (Sec. 4.3),
// FP64 on the GPU.
//
// Starts from the explicit preliminary factors (V^0, H^l, M^h, G^l, U^L of
// Sec. 3, built by build_explicit) and compresses every block to rank r0:
//   middle level (eq. KeqUCMRV): M~_p = C_p R_p^*, the middle factor becomes
//       the identity;
//   toward U^L (eq. GC), l = h+1..L: for output pair p the pencil
//       P = [G_{p,0} C_{q0}, G_{p,1} C_{q1}] (r x 2 r0) = C'_p [Gbar_{p,0}, Gbar_{p,1}];
//       Ubar = U^L C^L;
//   toward V^0 (eq. HR), l = h..1: for input pair q of level l-1, feeding
//       outputs p0, p1 through child c, the stacked pencil
//       Q = [R_{p0}^* H_{p0,c}; R_{p1}^* H_{p1,c}] (2 r0 x r) = [Hbar_{p0,c}; Hbar_{p1,c}] R'_q^*;
//       Vbar = R^0^* V^0.
// Each rank-r0 factorisation is the truncated SVD split as in eq.
// lowrankSVD, Z = (U0 S0^(1/2)) (S0^(1/2) V0^*).  The paper samples randomly
// for large blocks and notes that a direct SVD is as good for small r; here
// every block is at most 2r x r, so each thread computes a direct SVD by
// one-sided (Hestenes) Jacobi rotations in FP64: deterministic and accurate
// to rounding for singular values far below the largest.  The compressed
// factors have the explicit form's block shapes with r replaced by r0, so the
// explicit apply kernels run them unchanged.
#include <algorithm>
#include <cmath>

#include "ibf_internal.h"

namespace ibf {

typedef double2 cd;

constexpr int kOptMaxR = 12;   // blocks up to 2r x r = 24 x 12 per thread

__device__ __forceinline__ cd cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ cd cmul(cd a, cd b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cd cconj(cd a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ void cmac(cd& acc, cd a, cd b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// One-sided Jacobi on the n columns of X (m x n, column-major X[col * m + row]):
// rotations from the right make the columns mutually orthogonal, X <- X J,
// with J (n x n, column-major) accumulating them.  For the (p, q) column pair
// with Gram entries a = |x_p|^2, b = |x_q|^2, g = x_p^* x_q = |g| e^{i phi},
// the unitary G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] with t = tan(theta)
// the smaller root of t^2 + 2 tau t - 1 = 0, tau = (b - a) / (2 |g|), zeroes
// the pair's off-diagonal Gram entry.  Columns whose norm squared is below
// 1e-30 of the total count as zero.  At most 60 sweeps.
__device__ void jacobi_columns(cd* X, int m, int n, cd* J)
{
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) J[c * n + i] = make_double2(c == i ? 1.0 : 0.0, 0.0);
    double fro = 0.0;
    for (int e = 0; e < m * n; ++e) fro += X[e].x * X[e].x + X[e].y * X[e].y;
    const double small = 1e-30 * fro;
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rot = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                cd* xp = X + p * m;
                cd* xq = X + q * m;
                double a = 0.0, b = 0.0;
                cd g = cz();
                for (int i = 0; i < m; ++i) {
                    a += xp[i].x * xp[i].x + xp[i].y * xp[i].y;
                    b += xq[i].x * xq[i].x + xq[i].y * xq[i].y;
                    cmac(g, cconj(xp[i]), xq[i]);
                }
                const double ag = hypot(g.x, g.y);
                if (a <= small || b <= small || ag <= 1e-15 * sqrt(a * b)) continue;
                ++rot;
                const cd ec = make_double2(g.x / ag, -g.y / ag);   // e^{-i phi}
                const double tau = (b - a) / (2.0 * ag);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < m; ++i) {
                    const cd u = xp[i], v = cmul(ec, xq[i]);
                    xp[i] = make_double2(cs * u.x - sn * v.x, cs * u.y - sn * v.y);
                    xq[i] = make_double2(sn * u.x + cs * v.x, sn * u.y + cs * v.y);
                }
                cd* jp = J + p * n;
                cd* jq = J + q * n;
                for (int i = 0; i < n; ++i) {
                    const cd u = jp[i], v = cmul(ec, jq[i]);
                    jp[i] = make_double2(cs * u.x - sn * v.x, cs * u.y - sn * v.y);
                    jq[i] = make_double2(sn * u.x + cs * v.x, sn * u.y + cs * v.y);
                }
            }
        if (!rot) break;
    }
}

// indices of the k largest column norms of X (m x n), largest first, and
// those norms (the singular values)
__device__ void top_columns(const cd* X, int m, int n, int k, int* idx, double* sig)
{
    double nrm[kOptMaxR];
    for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += X[c * m + i].x * X[c * m + i].x + X[c * m + i].y * X[c * m + i].y;
        nrm[c] = sqrt(s);
    }
    bool used[kOptMaxR];
    for (int c = 0; c < n; ++c) used[c] = false;
    for (int j = 0; j < k; ++j) {
        int best = -1;
        for (int c = 0; c < n; ++c)
            if (!used[c] && (best < 0 || nrm[c] > nrm[best])) best = c;
        if (best < 0) {       // rank below k: pad with zero directions
            idx[j] = -1;
            sig[j] = 0.0;
            continue;
        }
        used[best] = true;
        idx[j] = best;
        sig[j] = nrm[best];
    }
}

// middle level: M~_p = C_p Rs_p, Rs = R^*; X = M~_p^* so that J holds the
// left singular vectors of M~_p and W = X J the scaled right ones
__global__ void kO_mid(const cd* M, cd* C, cd* Rs, cd* Mbar, int64_t N, int r, int r0)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= N) return;
    cd X[kOptMaxR * kOptMaxR], J[kOptMaxR * kOptMaxR];
    const cd* Mp = M + p * r * r;
    for (int t = 0; t < r; ++t)          // X[col t][row s] = conj(M[t][s])
        for (int s = 0; s < r; ++s) X[t * r + s] = cconj(Mp[t * r + s]);
    jacobi_columns(X, r, r, J);
    int idx[kOptMaxR];
    double sig[kOptMaxR];
    top_columns(X, r, r, r0, idx, sig);
    for (int k = 0; k < r0; ++k) {
        const double sq = sqrt(sig[k]), inv = sig[k] > 0.0 ? 1.0 / sq : 0.0;
        for (int t = 0; t < r; ++t) {
            const cd jv = idx[k] >= 0 ? J[idx[k] * r + t] : cz();
            C[(p * r + t) * r0 + k] = make_double2(jv.x * sq, jv.y * sq);
        }
        for (int s = 0; s < r; ++s) {
            const cd w = idx[k] >= 0 ? cconj(X[idx[k] * r + s]) : cz();
            Rs[(p * r0 + k) * r + s] = make_double2(w.x * inv, w.y * inv);
        }
        for (int k2 = 0; k2 < r0; ++k2) Mbar[(p * r0 + k) * r0 + k2] = make_double2(k == k2 ? 1.0 : 0.0, 0.0);
    }
}

// toward U^L at level l: output pair p = (i, j), inputs q0 + c = (i/2, 2j+c)
__global__ void kO_g(const cd* blk, const cd* Cin, cd* Cout, cd* Gbar, int L, int l, int64_t N, int r, int r0)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int64_t nj = 1LL << (L - l);
    const int64_t i = p >> (L - l), j = p & (nj - 1);
    const int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
    const int m = 2 * r0;
    cd X[2 * kOptMaxR * kOptMaxR], J[kOptMaxR * kOptMaxR];
    // P[t][c r0 + k] = sum_s blk[p][c][t][s] Cin[q_c][s][k];  X = P^* (2 r0 x r)
    for (int c = 0; c < 2; ++c)
        for (int t = 0; t < r; ++t) {
            const cd* row = blk + ((p * 2 + c) * r + t) * r;
            const cd* Cq = Cin + (q0 + c) * r * r0;
            for (int k = 0; k < r0; ++k) {
                cd acc = cz();
                for (int s = 0; s < r; ++s) cmac(acc, row[s], Cq[s * r0 + k]);
                X[t * m + c * r0 + k] = cconj(acc);
            }
        }
    jacobi_columns(X, m, r, J);
    int idx[kOptMaxR];
    double sig[kOptMaxR];
    top_columns(X, m, r, r0, idx, sig);
    for (int k = 0; k < r0; ++k) {
        const double sq = sqrt(sig[k]), inv = sig[k] > 0.0 ? 1.0 / sq : 0.0;
        for (int t = 0; t < r; ++t) {
            const cd jv = idx[k] >= 0 ? J[idx[k] * r + t] : cz();
            Cout[(p * r + t) * r0 + k] = make_double2(jv.x * sq, jv.y * sq);
        }
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < r0; ++s) {
                const cd w = idx[k] >= 0 ? cconj(X[idx[k] * m + c * r0 + s]) : cz();
                Gbar[((p * 2 + c) * r0 + k) * r0 + s] = make_double2(w.x * inv, w.y * inv);
            }
    }
}

// toward V^0 at level l: input pair q = (ip, C) of level l-1 feeds outputs
// p_a = (2 ip + a, C/2), a = 0, 1, through child c = C & 1
__global__ void kO_h(const cd* blk, const cd* Rsin, cd* Rsout, cd* Hbar, int L, int l, int64_t N, int r, int r0)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    const int64_t nj = 1LL << (L - l), nC = 2 * nj;
    const int64_t ip = q / nC, Cq = q % nC, j = Cq >> 1;
    const int c = (int)(Cq & 1);
    const int m = 2 * r0;
    cd X[2 * kOptMaxR * kOptMaxR], J[kOptMaxR * kOptMaxR];
    // Q[a r0 + k][s] = sum_t Rsin[p_a][k][t] blk[p_a][c][t][s];  X = Q (2 r0 x r)
    for (int a = 0; a < 2; ++a) {
        const int64_t pa = (2 * ip + a) * nj + j;
        const cd* B = blk + (pa * 2 + c) * r * r;
        const cd* R = Rsin + pa * r0 * r;
        for (int k = 0; k < r0; ++k)
            for (int s = 0; s < r; ++s) {
                cd acc = cz();
                for (int t = 0; t < r; ++t) cmac(acc, R[k * r + t], B[t * r + s]);
                X[s * m + a * r0 + k] = acc;
            }
    }
    jacobi_columns(X, m, r, J);
    int idx[kOptMaxR];
    double sig[kOptMaxR];
    top_columns(X, m, r, r0, idx, sig);
    for (int k = 0; k < r0; ++k) {
        const double sq = sqrt(sig[k]), inv = sig[k] > 0.0 ? 1.0 / sq : 0.0;
        for (int s = 0; s < r; ++s) {
            const cd jv = idx[k] >= 0 ? cconj(J[idx[k] * r + s]) : cz();
            Rsout[(q * r0 + k) * r + s] = make_double2(jv.x * sq, jv.y * sq);
        }
        for (int a = 0; a < 2; ++a) {
            const int64_t pa = (2 * ip + a) * nj + j;
            for (int k2 = 0; k2 < r0; ++k2) {
                const cd w = idx[k] >= 0 ? X[idx[k] * m + a * r0 + k2] : cz();
                Hbar[((pa * 2 + c) * r0 + k2) * r0 + k] = make_double2(w.x * inv, w.y * inv);
            }
        }
    }
}

// Ubar[n] = U[n] C^L_{leaf(n)}
__global__ void kO_u(const cd* U, const int32_t* leaf, const cd* C, cd* Ubar, int64_t nx, int r, int r0)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nx * r0) return;
    const int64_t n = e / r0;
    const int k = (int)(e % r0);
    const cd* Cl = C + (int64_t)leaf[n] * r * r0;
    cd acc = cz();
    for (int t = 0; t < r; ++t) cmac(acc, U[n * r + t], Cl[t * r0 + k]);
    Ubar[e] = acc;
}

// Vbar[k] = R^0_k^* V[k]
__global__ void kO_v(const cd* V, const cd* Rs, cd* Vbar, int64_t N, int r, int r0)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * r0) return;
    const int64_t k = e / r0;
    const int kk = (int)(e % r0);
    cd acc = cz();
    for (int t = 0; t < r; ++t) cmac(acc, Rs[(k * r0 + kk) * r + t], V[k * r + t]);
    Vbar[e] = acc;
}

static inline unsigned nbk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

int compress_optimal(ibf_plan* p, int r0, void* (*alloc)(ibf_plan*, size_t), void (*release)(ibf_plan*, void*))
{
    const int64_t N = p->N;
    const int r = p->r, L = p->L, h = p->h;
    const size_t c16 = sizeof(cd);
    cd* C = (cd*)alloc(p, c16 * N * r * r0);
    cd* C2 = (cd*)alloc(p, c16 * N * r * r0);
    cd* Rs = (cd*)alloc(p, c16 * N * r0 * r);
    cd* Rs2 = (cd*)alloc(p, c16 * N * r0 * r);
    cd* Mbar = (cd*)alloc(p, c16 * N * r0 * r0);
    cd* Ubar = (cd*)alloc(p, c16 * p->nx * r0);
    cd* Vbar = (cd*)alloc(p, c16 * N * r0);
    std::vector<void*> bar(L + 1, nullptr);
    for (int l = 1; l <= L; ++l) bar[l] = alloc(p, c16 * N * 2 * r0 * r0);
    for (void* q : {(void*)C, (void*)C2, (void*)Rs, (void*)Rs2, (void*)Mbar, (void*)Ubar, (void*)Vbar})
        if (!q) return set_error(IBF_ERR_OOM, "optimal IBF: factor allocation");
    for (int l = 1; l <= L; ++l)
        if (!bar[l]) return set_error(IBF_ERR_OOM, "optimal IBF: factor allocation");
    const int B = 64;
    kO_mid<<<nbk(N, B), B>>>((const cd*)p->eM, C, Rs, Mbar, N, r, r0);
    for (int l = h + 1; l <= L; ++l) {
        kO_g<<<nbk(N, B), B>>>((const cd*)p->eblk[l], C, C2, (cd*)bar[l], L, l, N, r, r0);
        std::swap(C, C2);
    }
    kO_u<<<nbk(p->nx * r0, 256), 256>>>((const cd*)p->eU, p->d_leaf, C, Ubar, p->nx, r, r0);
    for (int l = h; l >= 1; --l) {
        kO_h<<<nbk(N, B), B>>>((const cd*)p->eblk[l], Rs, Rs2, (cd*)bar[l], L, l, N, r, r0);
        std::swap(Rs, Rs2);
    }
    kO_v<<<nbk(N * r0, 256), 256>>>((const cd*)p->eV, Rs, Vbar, N, r, r0);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "optimal IBF compression");
    // the compressed factors replace the preliminary ones
    release(p, p->eV);
    release(p, p->eM);
    release(p, p->eU);
    for (int l = 1; l <= L; ++l) release(p, p->eblk[l]);
    for (void* q : {(void*)C, (void*)C2, (void*)Rs, (void*)Rs2}) release(p, q);
    p->eV = Vbar;
    p->eM = Mbar;
    p->eU = Ubar;
    for (int l = 1; l <= L; ++l) p->eblk[l] = bar[l];
    p->ra = r0;
    p->nnz = N * r0 + (int64_t)L * N * 2 * r0 * r0 + N * r0 * r0 + p->nx * r0;
    return IBF_OK;
}

// ---------------------------------------------------------------- sweep-in
//
// Sec. 4.3: after the sweep-out, the outer factors are compressed toward the
// middle.  G side: Ubar = Udot C^L per leaf, then for l = L..h+1, per input
// pair q of level l-1, [C_{p0} Gbar_{p0,c}; C_{p1} Gbar_{p1,c}] =
// [Gdot_{p0,c}; Gdot_{p1,c}] C_q.  H side: Vbar_j = A_j Vdot_j per frequency
// leaf, then for l = 1..h, per output pair p, [Hbar_{p,0} A_{q0},
// Hbar_{p,1} A_{q1}] = A_p [Hdot_{p,0}, Hdot_{p,1}] (A = R^*).  Middle:
// Mdot = C^h Mbar A^h with Mbar = I.  The rank of each split is the number
// of points the boxes hold, capped at r0 (K^G_l: the largest X-box count at
// level l; K^H_l = 2^l frequencies), so every split is exact.  Once a side's
// rank reaches r0 the remaining splits would only change bases: that side
// stops, merging its last C (or A) into the next level's blocks.

// per leaf i (n <= K < r0 points): X = Ubar_i^* (r0 x n); Ubar_i = J W^*
__global__ void kI_leaf_u(const cd* Ubar, const int32_t* off, cd* Ud, cd* C, int64_t N, int r0, int K)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n0 = off[i];
    const int n = min(off[i + 1] - n0, K);      // K bounds every leaf's count
    cd X[kOptMaxR * kOptMaxR], J[kOptMaxR * kOptMaxR];
    for (int a = 0; a < n; ++a)
        for (int s = 0; s < r0; ++s) X[a * r0 + s] = cconj(Ubar[(int64_t)(n0 + a) * r0 + s]);
    if (n > 0) jacobi_columns(X, r0, n, J);
    int idx[kOptMaxR];
    double sig[kOptMaxR];
    top_columns(X, r0, n, K, idx, sig);
    for (int k = 0; k < K; ++k) {
        const double sq = sqrt(sig[k]), inv = sig[k] > 0.0 ? 1.0 / sq : 0.0;
        for (int a = 0; a < n; ++a) {
            const cd jv = idx[k] >= 0 ? J[idx[k] * n + a] : cz();
            Ud[(int64_t)(n0 + a) * K + k] = make_double2(jv.x * sq, jv.y * sq);
        }
        for (int s = 0; s < r0; ++s) {
            const cd w = idx[k] >= 0 ? cconj(X[idx[k] * r0 + s]) : cz();
            C[(i * K + k) * r0 + s] = make_double2(w.x * inv, w.y * inv);
        }
    }
}

// G side, level l: input pair q of level l-1 feeds outputs p_a = (2 ip + a,
// C/2) through child c; Z = [C_{p0} B_{p0,c}; C_{p1} B_{p1,c}] (2 ko x r0)
// = [Gdot_{p0,c}; Gdot_{p1,c}] Cnew_q with Cnew_q ki x r0 and Gdot ko x ki
__global__ void kI_g(const cd* blk, const cd* Cin, cd* Cout, cd* Gd, int L, int l, int64_t N, int r0, int ko, int ki)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    const int64_t nj = 1LL << (L - l), nC = 2 * nj;
    const int64_t ip = q / nC, Cq = q % nC, j = Cq >> 1;
    const int c = (int)(Cq & 1);
    const int m = 2 * ko;
    cd X[2 * kOptMaxR * kOptMaxR], J[kOptMaxR * kOptMaxR];
    for (int a = 0; a < 2; ++a) {
        const int64_t pa = (2 * ip + a) * nj + j;
        const cd* B = blk + (pa * 2 + c) * r0 * r0;
        const cd* Cp = Cin + pa * ko * r0;
        for (int k = 0; k < ko; ++k)
            for (int s = 0; s < r0; ++s) {
                cd acc = cz();
                for (int t = 0; t < r0; ++t) cmac(acc, Cp[k * r0 + t], B[t * r0 + s]);
                X[s * m + a * ko + k] = acc;
            }
    }
    jacobi_columns(X, m, r0, J);
    int idx[kOptMaxR];
    double sig[kOptMaxR];
    top_columns(X, m, r0, ki, idx, sig);
    for (int k = 0; k < ki; ++k) {
        const double sq = sqrt(sig[k]), inv = sig[k] > 0.0 ? 1.0 / sq : 0.0;
        for (int s = 0; s < r0; ++s) {
            const cd jv = idx[k] >= 0 ? cconj(J[idx[k] * r0 + s]) : cz();
            Cout[(q * ki + k) * r0 + s] = make_double2(jv.x * sq, jv.y * sq);
        }
        for (int a = 0; a < 2; ++a) {
            const int64_t pa = (2 * ip + a) * nj + j;
            for (int k2 = 0; k2 < ko; ++k2) {
                const cd w = idx[k] >= 0 ? X[idx[k] * m + a * ko + k2] : cz();
                Gd[((pa * 2 + c) * ko + k2) * ki + k] = make_double2(w.x * inv, w.y * inv);
            }
        }
    }
}

// G side stops: Gdot_{p,c} = C_p B_{p,c} (ko x r0), one thread per entry
__global__ void kI_gmerge(const cd* blk, const cd* Cin, cd* Gd, int64_t N, int r0, int ko)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * 2 * ko * r0) return;
    const int s = (int)(e % r0), k = (int)((e / r0) % ko);
    const int64_t pc = e / ((int64_t)r0 * ko), p = pc >> 1;
    cd acc = cz();
    for (int t = 0; t < r0; ++t) cmac(acc, Cin[(p * ko + k) * r0 + t], blk[(pc * r0 + t) * r0 + s]);
    Gd[e] = acc;
}

// per frequency leaf j (one frequency): Vbar_j (r0 x 1) = A_j Vdot_j with
// sigma = |Vbar_j|, A_j = Vbar_j / sqrt(sigma), Vdot_j = sqrt(sigma)
__global__ void kI_leaf_v(const cd* Vbar, cd* Vd, cd* A, int64_t N, int r0)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s2 = 0.0;
    for (int t = 0; t < r0; ++t) s2 += Vbar[j * r0 + t].x * Vbar[j * r0 + t].x + Vbar[j * r0 + t].y * Vbar[j * r0 + t].y;
    const double sq = sqrt(sqrt(s2)), inv = s2 > 0.0 ? 1.0 / sq : 0.0;
    Vd[j] = make_double2(sq, 0.0);
    for (int t = 0; t < r0; ++t) A[j * r0 + t] = make_double2(Vbar[j * r0 + t].x * inv, Vbar[j * r0 + t].y * inv);
}

// H side, level l: output pair p = (i, j) reads q0 + c = (i/2, 2j+c);
// P = [B_{p,0} A_{q0}, B_{p,1} A_{q1}] (r0 x 2 ki) = Anew_p (r0 x ko) [Hdot_{p,0}, Hdot_{p,1}]
__global__ void kI_h(const cd* blk, const cd* Ain, cd* Aout, cd* Hd, int L, int l, int64_t N, int r0, int ki, int ko)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int64_t nj = 1LL << (L - l);
    const int64_t i = p >> (L - l), j = p & (nj - 1);
    const int64_t q0 = (i >> 1) * (2 * nj) + 2 * j;
    const int m = 2 * ki;
    cd X[2 * kOptMaxR * kOptMaxR], J[kOptMaxR * kOptMaxR];
    // X = P^* (2 ki x r0)
    for (int c = 0; c < 2; ++c)
        for (int t = 0; t < r0; ++t) {
            const cd* row = blk + ((p * 2 + c) * r0 + t) * r0;
            const cd* Aq = Ain + (q0 + c) * r0 * ki;
            for (int k = 0; k < ki; ++k) {
                cd acc = cz();
                for (int s = 0; s < r0; ++s) cmac(acc, row[s], Aq[s * ki + k]);
                X[t * m + c * ki + k] = cconj(acc);
            }
        }
    jacobi_columns(X, m, r0, J);
    int idx[kOptMaxR];
    double sig[kOptMaxR];
    top_columns(X, m, r0, ko, idx, sig);
    for (int k = 0; k < ko; ++k) {
        const double sq = sqrt(sig[k]), inv = sig[k] > 0.0 ? 1.0 / sq : 0.0;
        for (int t = 0; t < r0; ++t) {
            const cd jv = idx[k] >= 0 ? J[idx[k] * r0 + t] : cz();
            Aout[(p * r0 + t) * ko + k] = make_double2(jv.x * sq, jv.y * sq);
        }
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < ki; ++s) {
                const cd w = idx[k] >= 0 ? cconj(X[idx[k] * m + c * ki + s]) : cz();
                Hd[((p * 2 + c) * ko + k) * ki + s] = make_double2(w.x * inv, w.y * inv);
            }
    }
}

// H side stops: Hdot_{p,c} = B_{p,c} A_{q_c} (r0 x ki), one thread per entry
__global__ void kI_hmerge(const cd* blk, const cd* Ain, cd* Hd, int L, int l, int64_t N, int r0, int ki)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * 2 * r0 * ki) return;
    const int k = (int)(e % ki), t = (int)((e / ki) % r0);
    const int64_t pc = e / ((int64_t)ki * r0), p = pc >> 1;
    const int c = (int)(pc & 1);
    const int64_t nj = 1LL << (L - l);
    const int64_t i = p >> (L - l), j = p & (nj - 1);
    const int64_t q = (i >> 1) * (2 * nj) + 2 * j + c;
    cd acc = cz();
    for (int s = 0; s < r0; ++s) cmac(acc, blk[(pc * r0 + t) * r0 + s], Ain[(q * r0 + s) * ki + k]);
    Hd[e] = acc;
}

// Mdot_p = C^h_p A^h_p (kg x kh); a NULL side is the identity (its rank is r0)
__global__ void kI_mid(const cd* Cg, const cd* Ah, cd* Md, int64_t N, int r0, int kg, int kh)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * kg * kh) return;
    const int k2 = (int)(e % kh), k = (int)((e / kh) % kg);
    const int64_t p = e / ((int64_t)kg * kh);
    cd acc = cz();
    if (!Cg)
        acc = Ah[(p * r0 + k) * kh + k2];
    else if (!Ah)
        acc = Cg[(p * kg + k) * r0 + k2];
    else
        for (int s = 0; s < r0; ++s) cmac(acc, Cg[(p * kg + k) * r0 + s], Ah[(p * r0 + s) * kh + k2]);
    Md[e] = acc;
}

int sweep_in_optimal(ibf_plan* p, const std::vector<int32_t>& off, void* (*alloc)(ibf_plan*, size_t),
                     void (*release)(ibf_plan*, void*))
{
    const int64_t N = p->N;
    const int L = p->L, h = p->h, r0 = p->ra;
    const size_t c16 = sizeof(cd);
    // ranks: the largest point count of the X boxes of level l, and the 2^l
    // frequencies of the Omega boxes of level L - l, capped at r0
    std::vector<int> KG(L + 1, r0), KH(h + 1, r0);
    for (int l = h; l <= L; ++l) {
        const int64_t w = 1LL << (L - l);
        int64_t mx = 0;
        for (int64_t i = 0; i < (1LL << l); ++i) mx = std::max<int64_t>(mx, off[(i + 1) * w] - off[i * w]);
        KG[l] = (int)std::min<int64_t>(mx, r0);
    }
    for (int l = 0; l <= h; ++l) KH[l] = (int)std::min<int64_t>(1LL << std::min(l, 40), r0);
    const int B = 64;
    auto fail = [&](const char* what) { return set_error(IBF_ERR_OOM, what); };
    // a factor is freed only after the kernels that read it have finished
    auto drop = [&](void* q) {
        if (!q) return;
        cudaDeviceSynchronize();
        release(p, q);
    };
    // G side
    cd* C = nullptr;
    if (KG[L] < r0) {
        cd* Ud = (cd*)alloc(p, c16 * p->nx * KG[L]);
        C = (cd*)alloc(p, c16 * N * KG[L] * r0);
        if (!Ud || !C) return fail("sweep-in: factor allocation");
        kI_leaf_u<<<nbk(N, B), B>>>((const cd*)p->eU, p->d_off, Ud, C, N, r0, KG[L]);
        drop(p->eU);
        p->eU = Ud;
        for (int l = L; l > h; --l) {
            const int ko = KG[l], ki = KG[l - 1];
            if (ki < r0) {
                cd* Cn = (cd*)alloc(p, c16 * N * ki * r0);
                cd* Gd = (cd*)alloc(p, c16 * N * 2 * ko * ki);
                if (!Cn || !Gd) return fail("sweep-in: factor allocation");
                kI_g<<<nbk(N, B), B>>>((const cd*)p->eblk[l], C, Cn, Gd, L, l, N, r0, ko, ki);
                drop(C);
                drop(p->eblk[l]);
                p->eblk[l] = Gd;
                C = Cn;
            } else {
                cd* Gd = (cd*)alloc(p, c16 * N * 2 * ko * r0);
                if (!Gd) return fail("sweep-in: factor allocation");
                kI_gmerge<<<nbk(N * 2 * ko * r0, 256), 256>>>((const cd*)p->eblk[l], C, Gd, N, r0, ko);
                drop(C);
                C = nullptr;
                drop(p->eblk[l]);
                p->eblk[l] = Gd;
                break;
            }
        }
    }
    // H side
    cd* A = nullptr;
    if (KH[0] < r0) {
        cd* Vd = (cd*)alloc(p, c16 * N * KH[0]);
        A = (cd*)alloc(p, c16 * N * r0 * KH[0]);
        if (!Vd || !A) return fail("sweep-in: factor allocation");
        kI_leaf_v<<<nbk(N, 256), 256>>>((const cd*)p->eV, Vd, A, N, r0);
        drop(p->eV);
        p->eV = Vd;
        for (int l = 1; l <= h; ++l) {
            const int ki = KH[l - 1], ko = KH[l];
            if (ko < r0) {
                cd* An = (cd*)alloc(p, c16 * N * r0 * ko);
                cd* Hd = (cd*)alloc(p, c16 * N * 2 * ko * ki);
                if (!An || !Hd) return fail("sweep-in: factor allocation");
                kI_h<<<nbk(N, B), B>>>((const cd*)p->eblk[l], A, An, Hd, L, l, N, r0, ki, ko);
                drop(A);
                drop(p->eblk[l]);
                p->eblk[l] = Hd;
                A = An;
            } else {
                cd* Hd = (cd*)alloc(p, c16 * N * 2 * r0 * ki);
                if (!Hd) return fail("sweep-in: factor allocation");
                kI_hmerge<<<nbk(N * 2 * r0 * ki, 256), 256>>>((const cd*)p->eblk[l], A, Hd, L, l, N, r0, ki);
                drop(A);
                A = nullptr;
                drop(p->eblk[l]);
                p->eblk[l] = Hd;
                break;
            }
        }
    }
    // middle: either side that reached level h with rank below r0
    if (C || A) {
        cd* Md = (cd*)alloc(p, c16 * N * KG[h] * KH[h]);
        if (!Md) return fail("sweep-in: factor allocation");
        kI_mid<<<nbk(N * KG[h] * KH[h], 256), 256>>>(C, A, Md, N, r0, KG[h], KH[h]);
        drop(p->eM);
        p->eM = Md;
    }
    cudaError_t e = cudaDeviceSynchronize();
    drop(C);
    drop(A);
    if (e != cudaSuccess) return cuda_error(e, "optimal IBF sweep-in");
    p->rk_h = KH;
    p->rk_g = KG;
    int64_t nnz = N * KH[0] + N * (int64_t)KG[h] * KH[h] + p->nx * KG[L];
    for (int l = 1; l <= h; ++l) nnz += N * 2 * (int64_t)KH[l] * KH[l - 1];
    for (int l = h + 1; l <= L; ++l) nnz += N * 2 * (int64_t)KG[l] * KG[l - 1];
    p->nnz = nnz;
    return IBF_OK;
}

}  // namespace ibf
