// velsets.cuh -- compile-time velocity sets of Sec. 8 for the CUDA kernels.
//
// Each set is a type with constexpr accessors so that every sum over velocities in the kernels
// unrolls into straight-line code with the velocity components folded away.  The library's
// velocity order is its own: rest first, then opposite pairs next to each other.
//
// Coefficients are those of the general equilibrium of Sec. 5,
//   g_i^eq = ( a1 rho' + a2 theta' + b c_i.u' + |c_i|^2 (c1 rho' + c2 theta') / 2 ) f*_i,
// with theta' = ( (gamma - 1) sum_i (|c_i|^2 + beta_i) g_i / 2 - theta0 rho' ) / rho0.
// For the monoatomic sets the Sec. 4 equilibrium gives a1 = 1/rho0, a2 = -D/(2 theta0),
// b = 1/theta0, c1 = 0, c2 = 1/theta0^2, beta = 0 and gamma = (D + 2)/D.
#pragma once

#include "../../include/lee_lbm.h"

namespace lee {

// Velocity tables (x, y, z per row), shared by several sets.
struct Stencil {
    // rest, 6 faces, 12 edges, 8 corners; opposite pairs adjacent
    __host__ __device__ static constexpr int face(int k, int a) {
        constexpr int t[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        return t[k][a];
    }
    __host__ __device__ static constexpr int edge(int k, int a) {
        constexpr int t[12][3] = {{1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                  {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[k][a];
    }
    __host__ __device__ static constexpr int corner(int k, int a) {
        constexpr int t[8][3] = {{1, 1, 1},  {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
                                 {1, -1, 1}, {-1, 1, -1},  {-1, 1, 1}, {1, -1, -1}};
        return t[k][a];
    }
};

// Shell of velocity i: 0 rest, 1 face, 2 edge, 3 corner (|c|^2 = shell for these stencils).
// Weights f*, additional energies beta and all coefficients depend on the shell only.

struct D1Q3 {  // Sec. 8.1
    static constexpr int id = LEE_D1Q3, D = 1, Q = 3;
    static constexpr double rho0 = 1.0, theta0 = 1.0 / 3.0, gamma = 3.0;
    static constexpr double a1 = 1.0, a2 = -1.5, b = 3.0, c1 = 0.0, c2 = 9.0;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 1; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::face(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double betas(int) { return 0.0; }
};

struct D2Q5 {  // Sec. 8.2.1
    static constexpr int id = LEE_D2Q5, D = 2, Q = 5;
    static constexpr double rho0 = 1.0, theta0 = 0.25, gamma = 2.0;
    static constexpr double a1 = 1.0, a2 = -4.0, b = 4.0, c1 = 0.0, c2 = 16.0;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 1; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::face(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 0.5 : 0.125; }
    __host__ __device__ static constexpr double betas(int) { return 0.0; }
};

struct D2Q5Di {  // Sec. 8.2.2, diatomic: M = 3 degrees of freedom, gamma = 5/3
    static constexpr int id = LEE_D2Q5_DIATOMIC, D = 2, Q = 5;
    static constexpr double rho0 = 20.0 / 3.0, theta0 = 0.3, gamma = 5.0 / 3.0;
    static constexpr double a1 = 3.0 / 20.0, a2 = -5.0, b = 10.0 / 3.0, c1 = 0.0, c2 = 50.0 / 3.0;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 1; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::face(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 8.0 / 3.0 : 1.0; }
    __host__ __device__ static constexpr double betas(int s) { return s == 0 ? 0.0 : 0.5; }
};

struct D3Q7 {  // Sec. 8.3.1, theta0 = 1/5, alpha = 0
    static constexpr int id = LEE_D3Q7, D = 3, Q = 7;
    static constexpr double rho0 = 1.0, theta0 = 0.2, gamma = 5.0 / 3.0;
    static constexpr double a1 = 1.0, a2 = -7.5, b = 5.0, c1 = 0.0, c2 = 25.0;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 1; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::face(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 0.4 : 0.1; }
    __host__ __device__ static constexpr double betas(int) { return 0.0; }
};

struct D3Q9 {  // Sec. 8.3.1, theta0 = 3/5, alpha = 3/40: rest + 8 corners
    static constexpr int id = LEE_D3Q9, D = 3, Q = 9;
    static constexpr double rho0 = 1.0, theta0 = 0.6, gamma = 5.0 / 3.0;
    static constexpr double a1 = 1.0, a2 = -2.5, b = 5.0 / 3.0, c1 = 0.0, c2 = 25.0 / 9.0;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 3; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::corner(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 0.4 : 3.0 / 40.0; }
    __host__ __device__ static constexpr double betas(int) { return 0.0; }
};

struct D3Q13 {  // Sec. 8.3.1, theta0 = 2/5, alpha = 0: rest + 12 edges
    static constexpr int id = LEE_D3Q13, D = 3, Q = 13;
    static constexpr double rho0 = 1.0, theta0 = 0.4, gamma = 5.0 / 3.0;
    static constexpr double a1 = 1.0, a2 = -3.75, b = 2.5, c1 = 0.0, c2 = 6.25;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 2; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::edge(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 0.4 : 0.05; }
    __host__ __device__ static constexpr double betas(int) { return 0.0; }
};

struct D3Q19 {  // Sec. 8.3.1, theta0 = 3/10, alpha = 0: rest + 6 faces + 12 edges
    static constexpr int id = LEE_D3Q19, D = 3, Q = 19;
    static constexpr double rho0 = 1.0, theta0 = 0.3, gamma = 5.0 / 3.0;
    static constexpr double a1 = 1.0, a2 = -5.0, b = 10.0 / 3.0, c1 = 0.0, c2 = 100.0 / 9.0;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }
    __host__ __device__ static constexpr int c(int i, int a) {
        return i == 0 ? 0 : (i <= 6 ? Stencil::face(i - 1, a) : Stencil::edge(i - 7, a));
    }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 13.0 / 40.0 : (s == 1 ? 3.0 / 40.0 : 3.0 / 160.0); }
    __host__ __device__ static constexpr double betas(int) { return 0.0; }
};

struct D3Q7Di {  // Sec. 8.3.2, f1 = 5/42: diatomic, M = 5 degrees of freedom, gamma = 7/5
    static constexpr int id = LEE_D3Q7_DIATOMIC, D = 3, Q = 7;
    static constexpr double rho0 = 1.0, theta0 = 5.0 / 21.0, gamma = 1.4;
    static constexpr double a1 = 1.0, a2 = -10.5, b = 4.2, c1 = 0.0, c2 = 29.4;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 1; }
    __host__ __device__ static constexpr int c(int i, int a) { return i == 0 ? 0 : Stencil::face(i - 1, a); }
    __host__ __device__ static constexpr double fs(int s) { return s == 0 ? 2.0 / 7.0 : 5.0 / 42.0; }
    __host__ __device__ static constexpr double betas(int s) { return s == 0 ? 0.0 : 2.0 / 3.0; }
};

// Derived per-velocity quantities.
template <class S>
__host__ __device__ constexpr double f_of(int i) { return S::fs(S::shell(i)); }
template <class S>
__host__ __device__ constexpr double beta_of(int i) { return S::betas(S::shell(i)); }
template <class S>
__host__ __device__ constexpr int csq(int i) { return S::c(i, 0) * S::c(i, 0) + S::c(i, 1) * S::c(i, 1) + S::c(i, 2) * S::c(i, 2); }

// Calls fn(S{}) for the set with id `set`; returns false for an unknown id.
template <class Fn>
inline bool dispatch_set(int set, Fn &&fn) {
    switch (set) {
    case LEE_D1Q3: fn(D1Q3{}); return true;
    case LEE_D2Q5: fn(D2Q5{}); return true;
    case LEE_D2Q5_DIATOMIC: fn(D2Q5Di{}); return true;
    case LEE_D3Q7: fn(D3Q7{}); return true;
    case LEE_D3Q9: fn(D3Q9{}); return true;
    case LEE_D3Q13: fn(D3Q13{}); return true;
    case LEE_D3Q19: fn(D3Q19{}); return true;
    case LEE_D3Q7_DIATOMIC: fn(D3Q7Di{}); return true;
    default: return false;
    }
}

}  // namespace lee
