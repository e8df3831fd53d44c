/*
 * lee_stability.h -- von Neumann stability scan of the LBE update (Sec. 7, Theorem 1), on the GPU.
 *
 * Fourier transforming the update g(t+1, x + c_i) = H(tau) g(t, x) (Sec. 6, eq. "LBE linear
 * equation") gives g^(k, t+1) = Gamma(k) g^(k, t) with
 *     Gamma(k) = D(k) H(tau),   D_nn(k) = exp(-i k.c_n)      (lattice units, epsilon = 1).
 * Theorem 1 (Sec. 7): the scheme is L2-stable if, for every k with k_a in [-pi, pi], (1) Gamma is
 * regular, (2) its spectral radius is at most 1 and (3) the condition number of its eigenvector
 * matrix stays bounded.
 *
 * The scan evaluates these on the grid of m^D wave vectors
 *     k_a = 2 pi (j_a - m/2) / m,  j_a = 0 .. m-1,   point index j = j_x + m (j_y + m j_z),
 * one GPU thread per point, in FP64:
 *   lambda[j][n]  the q eigenvalues of Gamma(k) (re, im pairs), in no particular order;
 *   rho[j]        the spectral radius max_n |lambda_n| (condition 2);
 *   kappa[j]      condition 3, evaluated on the similar matrix Gamma_W = W^(1/2) Gamma W^(-1/2),
 *                 W = diag(1 / f*_n): the 2-norm condition number of its eigenvectors with unit
 *                 columns that are orthonormal within each cluster of eigenvalues closer than
 *                 `delta` (repeated eigenvalues -- the non-propagating entropy and vorticity
 *                 modes, at every k for tau = 1/2 -- leave the plain eigenvector matrix undefined).
 *                 The eigenvectors V of Gamma itself then satisfy
 *                 kappa_2(V) <= sqrt(max f* / min f*) kappa[j].  H is self-adjoint in the
 *                 W-weighted inner product, so Gamma_W = D(k) S with S symmetric, and at
 *                 tau = 1/2 Gamma_W is unitary for every set: kappa = 1;
 *   nu[j]         the normality defect ||G^H G - G G^H||_F / ||G||_F^2 of G = Gamma_W.
 * Condition 1 needs no scan: |det Gamma(k)| = |det H(tau)| = |1 - 1/tau|^(q - D - 2) for all k.
 *
 * Method per point: Householder reduction of Gamma_W to upper Hessenberg form; complex shifted QR
 * (Wilkinson shifts, deflation, at most 60 q iterations) for the eigenvalues; clusters by chained
 * distances below delta; for a single eigenvalue two rounds of inverse iteration with
 * (Gamma_W - lambda_c I), for a cluster of several the null space of (Gamma_W - lambda_c I)
 * (the eigenvectors of its Gram matrix for the smallest eigenvalues, by cyclic Jacobi); cyclic
 * Jacobi sweeps (at most 40 each) on U^H U for the extreme singular values of the eigenvector
 * matrix U.  A point whose QR iteration does not converge gets rho = kappa = NaN.
 *
 * H(tau) is built from the library's own folded collision coefficients, in the library's velocity
 * order (lee_velset_info).  The library computes Gamma; it does not decide stability.
 */
#ifndef LEE_STABILITY_H
#define LEE_STABILITY_H

#include <stdint.h>

#include "lee_lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* set: lee_velset; tau > 0 (tau < 1/2 is allowed here: it shows the instability);
 * m >= 1 with m^D <= 2^24; delta > 0 (1e-6 is a good choice for FP64);
 * lambda: device [m^D][q][2] doubles or NULL; rho: device [m^D] (required); kappa, nu: device
 * [m^D] or NULL; cuda_stream: the stream to run on (NULL = legacy default stream).
 * Asynchronous; allocates and frees one small device buffer (the q x q matrices) on the stream.
 * Returns LEE_ERR_INVALID_ARGUMENT for a bad argument, LEE_ERR_CUDA for a failed launch. */
lee_status lee_stability_scan(int32_t set, double tau, int32_t m, double delta, double *lambda, double *rho,
                              double *kappa, double *nu, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LEE_STABILITY_H */
