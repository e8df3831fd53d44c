// stability.cu -- von Neumann stability scan (include/lee_stability.h): one thread per wave
// vector, FP64 complex linear algebra on q x q matrices (q <= 19) held in the thread's local
// memory.  Every iteration below has a fixed upper bound.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/lee_stability.h"
#include "ops.cuh"

namespace lee {

SetConsts consts_for(int set, double scale);
void fold_coefficients(int set, bool scaled, double omega, double M[4][4], double N[4][4]);

namespace {

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx mk(double r, double i) { return cplx{r, i}; }
__device__ __forceinline__ cplx add(cplx a, cplx b) { return mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cplx sub(cplx a, cplx b) { return mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx mul(cplx a, cplx b) { return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re); }  // conj(a) b
__device__ __forceinline__ cplx scl(cplx a, double s) { return mk(a.re * s, a.im * s); }
__device__ __forceinline__ cplx conjg(cplx a) { return mk(a.re, -a.im); }
__device__ __forceinline__ double cabs(cplx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    const double d = abs2(b);
    return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__device__ __forceinline__ cplx csqrt(cplx z) {
    const double r = cabs(z);
    const double x = sqrt(0.5 * (r + fabs(z.re)));
    if (x == 0.0) return mk(0.0, 0.0);
    if (z.re >= 0.0) return mk(x, z.im / (2.0 * x));
    return mk(fabs(z.im) / (2.0 * x), z.im >= 0.0 ? x : -x);
}

constexpr int kQrIterPerEig = 60;
constexpr int kJacobiSweeps = 40;

struct ScanParams {
    int q, D, m;
    long long npts;
    double delta;
    const double *S;   // [q][q] symmetric: W^(1/2) H W^(-1/2)
    const double *S2;  // [q][q] S * S
    const int *c;      // [q][3]
    double *lambda, *rho, *kappa, *nu;
};

// Cyclic Jacobi on a Hermitian matrix B (at most kJacobiSweeps sweeps): B becomes diagonal with
// its eigenvalues; if V is given it starts as the identity and collects the eigenvectors (columns).
template <int Q>
__device__ void herm_jacobi(cplx (&B)[Q][Q], cplx (*V)[Q]) {
    if (V)
        for (int r = 0; r < Q; ++r)
            for (int c = 0; c < Q; ++c) V[r][c] = mk(r == c ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int r = 0; r < Q; ++r) {
            dia += B[r][r].re * B[r][r].re;
            for (int c = r + 1; c < Q; ++c) off += abs2(B[r][c]);
        }
        if (off <= 1e-32 * dia || off == 0.0) break;
        for (int pp = 0; pp < Q; ++pp)
            for (int rr = pp + 1; rr < Q; ++rr) {
                const cplx b = B[pp][rr];
                const double ab = cabs(b);
                if (ab == 0.0) continue;
                const double a = B[pp][pp].re, d = B[rr][rr].re;
                const cplx e = scl(b, 1.0 / ab);  // e^(i phi)
                const double tau = (d - a) / (2.0 * ab);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                // unitary on columns (pp, rr): [[cs, sn], [-sn conj(e), cs conj(e)]]
                for (int n = 0; n < Q; ++n) {
                    const cplx u = B[n][pp], w = B[n][rr];
                    B[n][pp] = sub(scl(u, cs), scl(mul(w, conjg(e)), sn));
                    B[n][rr] = add(scl(u, sn), scl(mul(w, conjg(e)), cs));
                }
                for (int n = 0; n < Q; ++n) {  // and its adjoint on rows (pp, rr)
                    const cplx u = B[pp][n], w = B[rr][n];
                    B[pp][n] = sub(scl(u, cs), scl(mul(e, w), sn));
                    B[rr][n] = add(scl(u, sn), scl(mul(e, w), cs));
                }
                B[pp][rr] = mk(0.0, 0.0);
                B[rr][pp] = mk(0.0, 0.0);
                B[pp][pp].im = 0.0;
                B[rr][rr].im = 0.0;
                if (V)
                    for (int n = 0; n < Q; ++n) {
                        const cplx u = V[n][pp], w = V[n][rr];
                        V[n][pp] = sub(scl(u, cs), scl(mul(w, conjg(e)), sn));
                        V[n][rr] = add(scl(u, sn), scl(mul(w, conjg(e)), cs));
                    }
            }
    }
}

template <int Q>
__global__ void __launch_bounds__(64) k_stability_scan(ScanParams p) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.npts) return;
    constexpr double kEps = 2.220446049250313e-16;
    // wave vector of point j
    double k[3] = {0.0, 0.0, 0.0};
    {
        long long r = j;
        for (int a = 0; a < p.D; ++a) {
            const int ja = (int)(r % p.m);
            r /= p.m;
            k[a] = 2.0 * 3.14159265358979323846 * (double)(ja - p.m / 2) / (double)p.m;
        }
    }
    cplx ph[Q];
    for (int n = 0; n < Q; ++n) {
        const double arg = -(k[0] * p.c[3 * n] + k[1] * p.c[3 * n + 1] + k[2] * p.c[3 * n + 2]);
        double sn, cs;
        sincos(arg, &sn, &cs);
        ph[n] = mk(cs, sn);
    }
    // G = D(k) S, kept; A = working copy
    cplx G[Q][Q], A[Q][Q];
    double gnorm2 = 0.0;
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) {
            G[r][c] = scl(ph[r], p.S[r * Q + c]);
            A[r][c] = G[r][c];
            gnorm2 += abs2(G[r][c]);
        }
    // normality defect: G^H G = S^2, (G G^H)_mn = ph_m conj(ph_n) (S^2)_mn
    if (p.nu) {
        double d2 = 0.0;
        for (int r = 0; r < Q; ++r)
            for (int c = 0; c < Q; ++c) {
                const double s2 = p.S2[r * Q + c];
                const cplx e = cmul(ph[c], ph[r]);  // ph_r conj(ph_c)
                d2 += s2 * s2 * abs2(sub(mk(1.0, 0.0), e));
            }
        p.nu[j] = sqrt(d2) / gnorm2;
    }

    // --- Householder reduction to upper Hessenberg form
    for (int col = 0; col + 2 < Q; ++col) {
        double alpha2 = 0.0;
        for (int i = col + 1; i < Q; ++i) alpha2 += abs2(A[i][col]);
        const double alpha = sqrt(alpha2);
        if (alpha == 0.0) continue;
        const cplx x0 = A[col + 1][col];
        const double ax0 = cabs(x0);
        const cplx phase = ax0 > 0.0 ? scl(x0, 1.0 / ax0) : mk(1.0, 0.0);
        cplx v[Q];
        for (int i = 0; i < Q; ++i) v[i] = mk(0.0, 0.0);
        for (int i = col + 1; i < Q; ++i) v[i] = A[i][col];
        v[col + 1] = add(v[col + 1], scl(phase, alpha));
        double vn2 = 0.0;
        for (int i = col + 1; i < Q; ++i) vn2 += abs2(v[i]);
        const double f = 2.0 / vn2;
        for (int c = col; c < Q; ++c) {  // A <- (I - f v v^H) A
            cplx s = mk(0.0, 0.0);
            for (int i = col + 1; i < Q; ++i) s = add(s, cmul(v[i], A[i][c]));
            for (int i = col + 1; i < Q; ++i) A[i][c] = sub(A[i][c], scl(mul(v[i], s), f));
        }
        for (int r = 0; r < Q; ++r) {  // A <- A (I - f v v^H)
            cplx s = mk(0.0, 0.0);
            for (int i = col + 1; i < Q; ++i) s = add(s, mul(A[r][i], v[i]));
            for (int i = col + 1; i < Q; ++i) A[r][i] = sub(A[r][i], scl(mul(s, conjg(v[i])), f));
        }
        for (int i = col + 2; i < Q; ++i) A[i][col] = mk(0.0, 0.0);
    }

    // --- shifted QR on the Hessenberg matrix (eigenvalues only)
    bool ok = true;
    {
        int hi = Q - 1, it = 0, total = 0;
        while (hi > 0) {
            if (++total > kQrIterPerEig * Q) {
                ok = false;
                break;
            }
            int l = hi;
            while (l > 0 && cabs(A[l][l - 1]) > kEps * (cabs(A[l][l]) + cabs(A[l - 1][l - 1]))) --l;
            if (l > 0) A[l][l - 1] = mk(0.0, 0.0);
            if (l == hi) {  // A[hi][hi] has converged
                --hi;
                it = 0;
                continue;
            }
            ++it;
            const cplx a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
            cplx mu;
            if (it % 11 == 10) {  // exceptional shift
                mu = add(d, mk(cabs(c), 0.0));
            } else {  // Wilkinson: the eigenvalue of the trailing 2 x 2 block closer to d
                const cplx half = scl(sub(a, d), 0.5);
                const cplx disc = csqrt(add(mul(half, half), mul(b, c)));
                const cplx m1 = add(scl(add(a, d), 0.5), disc), m2 = sub(scl(add(a, d), 0.5), disc);
                mu = cabs(sub(m1, d)) < cabs(sub(m2, d)) ? m1 : m2;
            }
            for (int i = l; i <= hi; ++i) A[i][i] = sub(A[i][i], mu);
            cplx gc[Q], gs[Q];  // rotation kk: [x; y] -> [conj(gc) x + conj(gs) y; -gs x + gc y]
            for (int kk = l; kk < hi; ++kk) {
                const cplx x = A[kk][kk], y = A[kk + 1][kk];
                const double r = sqrt(abs2(x) + abs2(y));
                if (r == 0.0) {
                    gc[kk] = mk(1.0, 0.0);
                    gs[kk] = mk(0.0, 0.0);
                    continue;
                }
                gc[kk] = scl(x, 1.0 / r);
                gs[kk] = scl(y, 1.0 / r);
                for (int cc = kk; cc <= hi; ++cc) {
                    const cplx u = A[kk][cc], w = A[kk + 1][cc];
                    A[kk][cc] = add(cmul(gc[kk], u), cmul(gs[kk], w));
                    A[kk + 1][cc] = sub(mul(gc[kk], w), mul(gs[kk], u));
                }
            }
            for (int kk = l; kk < hi; ++kk) {  // A <- A G_kk^H on columns kk, kk+1
                const int rmax = kk + 1;
                for (int r = l; r <= rmax; ++r) {
                    const cplx u = A[r][kk], w = A[r][kk + 1];
                    A[r][kk] = add(mul(u, gc[kk]), mul(w, gs[kk]));
                    A[r][kk + 1] = sub(mul(w, conjg(gc[kk])), mul(u, conjg(gs[kk])));
                }
            }
            for (int i = l; i <= hi; ++i) A[i][i] = add(A[i][i], mu);
        }
    }
    cplx lam[Q];
    double rho = 0.0;
    for (int n = 0; n < Q; ++n) {
        lam[n] = A[n][n];
        rho = fmax(rho, cabs(lam[n]));
    }
    if (p.lambda) {
        for (int n = 0; n < Q; ++n) {
            p.lambda[(j * Q + n) * 2] = lam[n].re;
            p.lambda[(j * Q + n) * 2 + 1] = lam[n].im;
        }
    }
    p.rho[j] = ok ? rho : nan("");
    if (!p.kappa) return;
    if (!ok) {
        p.kappa[j] = nan("");
        return;
    }

    // --- clusters: chained distances below delta (union-find on q points)
    int parent[Q];
    for (int n = 0; n < Q; ++n) parent[n] = n;
    auto find = [&](int x) {
        for (int g = 0; g < Q && parent[x] != x; ++g) x = parent[x];
        return x;
    };
    for (int a = 0; a < Q; ++a)
        for (int b = a + 1; b < Q; ++b)
            if (cabs(sub(lam[a], lam[b])) < p.delta) {
                const int ra = find(a), rb = find(b);
                if (ra != rb) parent[rb < ra ? ra : rb] = rb < ra ? rb : ra;  // the smaller root wins
            }

    // --- per cluster, an orthonormal basis of its eigenspace
    cplx U[Q][Q], V[Q][Q];
    int ncol = 0;
    const double gscale = sqrt(gnorm2);
    for (int root = 0; root < Q; ++root) {
        if (find(root) != root) continue;
        int mc = 0;
        cplx lc = mk(0.0, 0.0);
        for (int n = 0; n < Q; ++n)
            if (find(n) == root) {
                ++mc;
                lc = add(lc, lam[n]);
            }
        lc = scl(lc, 1.0 / mc);
        if (mc > 1) {
            // several eigenvalues: the eigenspace is the null space of (G - lc I), spanned by the
            // eigenvectors of (G - lc I)^H (G - lc I) for its mc smallest eigenvalues (Jacobi); a
            // block inverse iteration would collapse onto one direction through the mc tiny pivots
            for (int r = 0; r < Q; ++r)
                for (int c = 0; c < Q; ++c) {
                    cplx acc = mk(0.0, 0.0);
                    for (int n = 0; n < Q; ++n) {
                        const cplx gr = n == r ? sub(G[n][r], lc) : G[n][r];
                        const cplx gc = n == c ? sub(G[n][c], lc) : G[n][c];
                        acc = add(acc, cmul(gr, gc));
                    }
                    A[r][c] = acc;
                }
            herm_jacobi<Q>(A, V);
            bool taken[Q];
            for (int n = 0; n < Q; ++n) taken[n] = false;
            for (int t = 0; t < mc; ++t) {
                int best = -1;
                for (int n = 0; n < Q; ++n)
                    if (!taken[n] && (best < 0 || A[n][n].re < A[best][best].re)) best = n;
                taken[best] = true;
                for (int n = 0; n < Q; ++n) U[n][ncol + t] = V[n][best];
            }
            ncol += mc;
            continue;
        }
        // one eigenvalue: inverse iteration with (G - lc I), LU with partial pivoting in A; a tiny
        // pivot is lifted to eps ||G||
        int piv[Q];
        for (int r = 0; r < Q; ++r)
            for (int c = 0; c < Q; ++c) A[r][c] = r == c ? sub(G[r][c], lc) : G[r][c];
        for (int c = 0; c < Q; ++c) {
            int pr = c;
            double best = cabs(A[c][c]);
            for (int r = c + 1; r < Q; ++r)
                if (cabs(A[r][c]) > best) {
                    best = cabs(A[r][c]);
                    pr = r;
                }
            piv[c] = pr;
            if (pr != c)
                for (int cc = 0; cc < Q; ++cc) {
                    const cplx t = A[c][cc];
                    A[c][cc] = A[pr][cc];
                    A[pr][cc] = t;
                }
            if (cabs(A[c][c]) < kEps * gscale) A[c][c] = mk(kEps * gscale, 0.0);
            for (int r = c + 1; r < Q; ++r) {
                const cplx f = cdiv(A[r][c], A[c][c]);
                A[r][c] = f;
                for (int cc = c + 1; cc < Q; ++cc) A[r][cc] = sub(A[r][cc], mul(f, A[c][cc]));
            }
        }
        // a fixed generic start vector, two rounds of x <- (G - lc I)^(-1) x, normalised
        for (int t = 0; t < mc; ++t)
            for (int n = 0; n < Q; ++n) {
                double sn, cs;
                sincos(1.0 + 0.754877666 * n + 2.2360679 * t + 0.31 * n * t, &sn, &cs);
                U[n][ncol + t] = mk(cs, 0.5 * sn);
            }
        for (int round = 0; round < 2; ++round) {
            for (int t = 0; t < mc; ++t) {
                cplx x[Q];
                for (int n = 0; n < Q; ++n) x[n] = U[n][ncol + t];
                for (int c = 0; c < Q; ++c) {  // apply the row swaps, then L, then U
                    const cplx tmp = x[c];
                    x[c] = x[piv[c]];
                    x[piv[c]] = tmp;
                }
                for (int r = 1; r < Q; ++r)
                    for (int c = 0; c < r; ++c) x[r] = sub(x[r], mul(A[r][c], x[c]));
                for (int r = Q - 1; r >= 0; --r) {
                    for (int c = r + 1; c < Q; ++c) x[r] = sub(x[r], mul(A[r][c], x[c]));
                    x[r] = cdiv(x[r], A[r][r]);
                }
                for (int n = 0; n < Q; ++n) U[n][ncol + t] = x[n];
            }
            for (int t = 0; t < mc; ++t) {  // modified Gram-Schmidt, twice
                for (int pass = 0; pass < 2; ++pass)
                    for (int s = 0; s < t; ++s) {
                        cplx d = mk(0.0, 0.0);
                        for (int n = 0; n < Q; ++n) d = add(d, cmul(U[n][ncol + s], U[n][ncol + t]));
                        for (int n = 0; n < Q; ++n) U[n][ncol + t] = sub(U[n][ncol + t], mul(U[n][ncol + s], d));
                    }
                double nn = 0.0;
                for (int n = 0; n < Q; ++n) nn += abs2(U[n][ncol + t]);
                const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
                for (int n = 0; n < Q; ++n) U[n][ncol + t] = scl(U[n][ncol + t], inv);
            }
        }
        ncol += mc;
    }

    // --- kappa_2(U) from the eigenvalues of the Hermitian B = U^H U (cyclic Jacobi), in A
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) {
            cplx s = mk(0.0, 0.0);
            for (int n = 0; n < Q; ++n) s = add(s, cmul(U[n][r], U[n][c]));
            A[r][c] = s;
        }
    herm_jacobi<Q>(A, nullptr);
    double emax = 0.0, emin = INFINITY;
    for (int r = 0; r < Q; ++r) {
        emax = fmax(emax, A[r][r].re);
        emin = fmin(emin, A[r][r].re);
    }
    p.kappa[j] = emin > 0.0 ? sqrt(emax / emin) : INFINITY;
}

}  // namespace
}  // namespace lee

using namespace lee;

extern "C" lee_status lee_stability_scan(int32_t set, double tau, int32_t m, double delta, double *lambda, double *rho,
                                         double *kappa, double *nu, void *cuda_stream) {
    const SetOps *o = set_ops(set);
    if (!o || !rho || !(tau > 0.0) || !std::isfinite(tau) || m < 1 || !(delta > 0.0)) return LEE_ERR_INVALID_ARGUMENT;
    long long npts = 1;
    for (int a = 0; a < o->D; ++a) {
        npts *= m;
        if (npts > (1LL << 24)) return LEE_ERR_INVALID_ARGUMENT;
    }
    const int q = o->Q;
    // H(tau) from the folded collision coefficients (kernels.cuh, CollideCoef):
    // H_ij = (1 - w) delta_ij + M[t][s] + N[t][s] c_i.c_j, t = shell(i), s = shell(j);
    // S = W^(1/2) H W^(-1/2), W = diag(1 / f*): S_ij = H_ij sqrt(f*_j / f*_i)
    const double omega = 1.0 / tau;
    double M[4][4], N[4][4];
    fold_coefficients(set, false, omega, M, N);
    const SetConsts k = consts_for(set, 1.0);
    const size_t qq = (size_t)q * q;
    double hbuf[2 * 19 * 19];
    int cbuf[19 * 3];
    double *S = hbuf, *S2 = hbuf + qq;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) cbuf[3 * i + a] = o->c[i][a];
        for (int jj = 0; jj < q; ++jj) {
            const int t = o->shell[i], s = o->shell[jj];
            const double cc = (double)(o->c[i][0] * o->c[jj][0] + o->c[i][1] * o->c[jj][1] + o->c[i][2] * o->c[jj][2]);
            const double h = (i == jj ? 1.0 - omega : 0.0) + M[t][s] + N[t][s] * cc;
            S[i * q + jj] = h * std::sqrt(k.f[s] / k.f[t]);
        }
    }
    for (int i = 0; i < q; ++i)
        for (int jj = 0; jj < q; ++jj) {
            double acc = 0.0;
            for (int l = 0; l < q; ++l) acc += S[i * q + l] * S[l * q + jj];
            S2[i * q + jj] = acc;
        }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void *dbuf = nullptr;
    const size_t bytes = sizeof(double) * 2 * qq + sizeof(int) * 3 * (size_t)q;
    if (cudaMallocAsync(&dbuf, bytes, st) != cudaSuccess) return LEE_ERR_CUDA;
    cudaError_t e = cudaMemcpyAsync(dbuf, hbuf, sizeof(double) * 2 * qq, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char *>(dbuf) + sizeof(double) * 2 * qq, cbuf, sizeof(int) * 3 * (size_t)q,
                            cudaMemcpyHostToDevice, st);
    ScanParams p;
    p.q = q;
    p.D = o->D;
    p.m = m;
    p.npts = npts;
    p.delta = delta;
    p.S = static_cast<const double *>(dbuf);
    p.S2 = p.S + qq;
    p.c = reinterpret_cast<const int *>(static_cast<const char *>(dbuf) + sizeof(double) * 2 * qq);
    p.lambda = lambda;
    p.rho = rho;
    p.kappa = kappa;
    p.nu = nu;
    const unsigned blocks = (unsigned)((npts + 63) / 64);
    if (e == cudaSuccess) {
        switch (q) {
        case 3: k_stability_scan<3><<<blocks, 64, 0, st>>>(p); break;
        case 5: k_stability_scan<5><<<blocks, 64, 0, st>>>(p); break;
        case 7: k_stability_scan<7><<<blocks, 64, 0, st>>>(p); break;
        case 9: k_stability_scan<9><<<blocks, 64, 0, st>>>(p); break;
        case 13: k_stability_scan<13><<<blocks, 64, 0, st>>>(p); break;
        case 19: k_stability_scan<19><<<blocks, 64, 0, st>>>(p); break;
        default: e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    // the copies read host stack memory: wait for them before returning
    const cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFreeAsync(dbuf, st);
    if (e != cudaSuccess || e2 != cudaSuccess) return LEE_ERR_CUDA;
    return LEE_OK;
}
