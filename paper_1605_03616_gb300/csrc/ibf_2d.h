// 2D multiscale IBF (Sec. 5): shared declarations of the construction and
// apply translation units.
#pragma once

#include <vector>

#include "ibf_internal.h"

namespace ibf {

// One ring of the corona decomposition: the 12 outer boxes (side m) of the
// 4 x 4 partition of S_t = [-n/2^(t+1), n/2^(t+1))^2.  Every box runs its own
// 2D butterfly of depth Lq = log2 m (switch level hq) against the whole X
// grid; the 12 boxes of a ring share every launch.
struct Ring2D {
    int m = 0, Lq = 0, hq = 0;
    double q1[12], q2[12];            // lower corners of the boxes
    // tables, box-major (box stride in elements given by the *_stride fields)
    void* V = nullptr;                // [box][m*m leaves][r2]
    std::vector<void*> D;             // level l = 1..Lq: [box][4^l][4^(Lq-l+1)][r2]
    void* M = nullptr;                // [box][m*m pairs][r2][r2]
    void* uph = nullptr;              // [box][nx] e(Phi(x_n, c_Q))
    void* lw = nullptr;               // [n/m][r] Lagrange weights of in-leaf offsets (real)
    int64_t v_stride = 0, d_stride = 0, m_stride = 0;
};

struct Plan2D {
    int n = 0;                        // grid side, N = n*n
    int center = 0;                   // side of the directly summed centre square
    std::vector<Ring2D> rings;
    void* KC = nullptr;               // [nx][center^2] centre kernel e(Phi(x_n, xi_k))
    void* ws[2] = {nullptr, nullptr}; // ring workspace: [box][m*m][r2][nrhs]
    size_t ws_elems = 0;              // elements per buffer
};

int build_2d(ibf_plan* p);
int apply_2d(ibf_plan* p, const void* g, void* u, int nrhs, cudaStream_t st);
int apply_2d_adjoint(ibf_plan* p, const void* y, void* g, int nrhs, cudaStream_t st);
int launches_2d(const ibf_plan* p);

}  // namespace ibf
