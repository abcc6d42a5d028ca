// Device helpers for the theta-dependent coefficients of the model
// (assembly and its derivatives in the adjoint gradient).
#pragma once

// M^{-1} entry [row][col] from lambda: unit lower triangular, -lambda below
// the diagonal ordered sub-diagonal by sub-diagonal (offset 1 first, top to
// bottom); for nv = 3 this reproduces the mixing matrix of Eq. 5.
static __device__ __forceinline__ double minv_entry(const double* lam, int nv, int row, int col) {
    if (row == col) return 1.0;
    if (row < col) return 0.0;
    const int off = row - col;
    int k = 0;
    for (int o = 1; o < off; ++o) k += nv - o;
    k += col;   // position within sub-diagonal `off` is the column index
    return -lam[k];
}

// Position (row, col) of lambda_l in M^{-1}.
static __device__ __forceinline__ void lambda_position(int nv, int l, int* row, int* col) {
    int k = 0;
    for (int off = 1; off < nv; ++off)
        for (int v = off; v < nv; ++v, ++k)
            if (k == l) {
                *row = v;
                *col = v - off;
                return;
            }
    *row = -1;
    *col = -1;
}

// Stationary unit-variance AR(1) precision entry Q_t[ti][tj].
static __device__ __forceinline__ double ar1_entry(double rho, int nt, int ti, int tj) {
    if (nt == 1) return 1.0;
    const double inv = 1.0 / (1.0 - rho * rho);
    if (ti == tj) return ((ti == 0 || ti == nt - 1) ? 1.0 : 1.0 + rho * rho) * inv;
    if (ti - tj == 1 || tj - ti == 1) return -rho * inv;
    return 0.0;
}

// d Q_t[ti][tj] / d rho.
static __device__ __forceinline__ double ar1_drho(double rho, int nt, int ti, int tj) {
    if (nt == 1) return 0.0;
    const double den = (1.0 - rho * rho) * (1.0 - rho * rho);
    if (ti == tj) return ((ti == 0 || ti == nt - 1) ? 2.0 * rho : 4.0 * rho) / den;
    if (ti - tj == 1 || tj - ti == 1) return -(1.0 + rho * rho) / den;
    return 0.0;
}
