/* RCLUPP through the C ABI alone (no Python, no PyTorch): a seeded 3000 x 24
 * test matrix X = U W D (U uniform in [-1, 1], W unit upper triangular with
 * off-diagonal entries in [-0.1, 0.1], D = diag(10^(-5 j / (n - 1))), so
 * kappa_2(X) is about 1e5) is built on the host, copied to the device with
 * the CUDA runtime, factored by rclupp_factor, rclupp_r_factor,
 * cholqr2_factor and lc2_factor, and checked on the host:
 * ||Q^T Q - I||_F and ||X - Q R||_F / ||X||_F at most 1e-13, R upper
 * triangular with a positive diagonal.  Prints "ok" and returns 0 on
 * success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "rclupp.h"

static uint64_t lcg_state = 20241206u;
static double uniform01(void)
{
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg_state >> 11) * 0x1p-53;
}

static void make_x(int64_t m, int64_t n, double *X)
{
    double *U = malloc(sizeof(double) * (size_t)(m * n));
    double *W = calloc((size_t)(n * n), sizeof(double));
    for (int64_t i = 0; i < m * n; ++i) U[i] = 2.0 * uniform01() - 1.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t k = 0; k < j; ++k) W[k + j * n] = 0.1 * (2.0 * uniform01() - 1.0);
        W[j + j * n] = 1.0;
    }
    for (int64_t j = 0; j < n; ++j) {
        const double d = pow(10.0, -5.0 * (double)j / (double)(n - 1));
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t k = 0; k <= j; ++k) s += U[i + k * m] * W[k + j * n];
            X[i + j * m] = s * d;
        }
    }
    free(U);
    free(W);
}

static int check(const char *name, int64_t m, int64_t n, const double *X, const double *Q,
                 const double *R)
{
    double orth = 0.0, res = 0.0, xn = 0.0;
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = 0; b < n; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) s += Q[i + a * m] * Q[i + b * m];
            s -= (a == b) ? 1.0 : 0.0;
            orth += s * s;
        }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t k = 0; k <= j; ++k) s += Q[i + k * m] * R[k + j * n];
            const double d = X[i + j * m] - s;
            res += d * d;
            xn += X[i + j * m] * X[i + j * m];
        }
    orth = sqrt(orth);
    res = sqrt(res / xn);
    int upper = 1;
    for (int64_t j = 0; j < n; ++j) {
        if (!(R[j + j * n] > 0.0)) upper = 0;
        for (int64_t i = j + 1; i < n; ++i)
            if (R[i + j * n] != 0.0) upper = 0;
    }
    printf("%-8s orth %.2e  res %.2e  %s\n", name, orth, res, upper ? "R upper, diag > 0" : "R BAD");
    return orth <= 1e-13 && res <= 1e-13 && upper;
}

int main(void)
{
    const int64_t m = 3000, n = 24;
    const size_t xb = sizeof(double) * (size_t)(m * n), rb = sizeof(double) * (size_t)(n * n);
    double *X = malloc(xb), *Q = malloc(xb), *R = malloc(rb);
    make_x(m, n, X);
    double *dX, *dQ, *dR;
    if (cudaMalloc((void **)&dX, xb) != cudaSuccess || cudaMalloc((void **)&dQ, xb) != cudaSuccess ||
        cudaMalloc((void **)&dR, rb) != cudaSuccess) {
        printf("cudaMalloc failed\n");
        return 2;
    }
    cudaMemcpy(dX, X, xb, cudaMemcpyHostToDevice);
    rclupp_handle_t h;
    if (rclupp_create(&h, NULL) != RCLUPP_OK) {
        printf("rclupp_create failed\n");
        return 2;
    }
    rclupp_opts_t o = {0};
    o.kind = RCLUPP_SKETCH_GAUSSIAN;
    o.s = 2 * n;
    o.zeta = 8;
    o.seed = 7;
    o.prec = RCLUPP_PREC_FP64;
    int ok = 1;
    for (int a = 0; a < 4; ++a) {
        rclupp_info_t info;
        rclupp_status_t st;
        const char *name;
        switch (a) {
            case 0: name = "rclupp"; st = rclupp_factor(h, m, n, dX, m, &o, dQ, m, dR, n, &info); break;
            case 1: name = "rcluppr"; st = rclupp_r_factor(h, m, n, dX, m, &o, dQ, m, dR, n, &info); break;
            case 2: name = "cholqr2"; st = cholqr2_factor(h, m, n, dX, m, dQ, m, dR, n, &info); break;
            default: name = "lc2"; st = lc2_factor(h, m, n, dX, m, dQ, m, dR, n, &info); break;
        }
        if (st != RCLUPP_OK) {
            printf("%s: %s\n", name, rclupp_status_string(st));
            ok = 0;
            continue;
        }
        cudaMemcpy(Q, dQ, xb, cudaMemcpyDeviceToHost);
        cudaMemcpy(R, dR, rb, cudaMemcpyDeviceToHost);
        ok &= check(name, m, n, X, Q, R);
    }
    rclupp_destroy(h);
    cudaFree(dX);
    cudaFree(dQ);
    cudaFree(dR);
    free(X);
    free(Q);
    free(R);
    printf(ok ? "ok\n" : "FAILED\n");
    return ok ? 0 : 1;
}
