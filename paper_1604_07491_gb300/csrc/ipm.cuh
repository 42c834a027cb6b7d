// ipm.cuh -- drivers shared by the C ABI.
#pragma once
#include "lpk_internal.cuh"

// Krylov solve of the row-scaled system for right-hand side f (sweep order);
// scale_rows must have been called for the current d2.  dy (m, sweep order)
// and dw (n) are unscaled outputs; tmp_m is an m-vector of scratch.
lpk_status ls_solve_scaled(lpk_ctx *ctx, DevProblem &P, const double *r, const double *f, int ell, double omega,
                           int precision, double tol, int maxit, double *dy, double *dw, double *tmp_m,
                           KrylovResult *kr);
lpk_status ne_solve_scaled(lpk_ctx *ctx, DevProblem &P, const double *f, int ell, double omega, int solver,
                           int precision, double tol, int maxit, double *dy, double *dw, double *tmp_m,
                           KrylovResult *kr);

// Algorithm 1 on device vectors in the input numbering.
lpk_status lp_solve_dev(lpk_ctx *ctx, DevProblem &P, const double *b_in, const double *c_in,
                        const lpk_options &o, double *x_in, double *y_in, double *s_in, lpk_info &info);
