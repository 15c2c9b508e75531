/* End-to-end use of the C-ABI from plain C (no Python): a 300 x 200 CSR
 * matrix with one entry per row whose singular values are known exactly,
 * created from host arrays, solved for the k = 5 largest triplets into host
 * outputs, then checked; plus the error paths a C caller sees.
 * Exit status 0 on success; prints what it found. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "svdsc.h"

#define M 300
#define N 200
#define K 5

int main(void)
{
    /* row i (< N) holds d_i at column i; rows N..M-1 are empty: sigma = |d_i| */
    static int64_t row_ptr[M + 1];
    static int32_t col[N];
    static double val[N], S[K], U[M * K], V[N * K], res[K];
    for (int i = 0; i <= M; i++) row_ptr[i] = i < N ? i : N;
    for (int i = 0; i < N; i++) {
        col[i] = (i * 7) % N;                               /* a permutation of the columns */
        val[i] = (i % 2 ? -1.0 : 1.0) * (1.0 + 0.01 * i);   /* |d| = 1 .. 2.99, distinct */
    }
    svdsc_matrix A = {0};
    A.format = SVDSC_CSR;
    A.index_base = 0;
    A.m = M;
    A.n = N;
    A.row_ptr = row_ptr;
    A.col_idx = col;
    A.values = val;
    A.value_type = SVDSC_F64;
    A.on_device = 0;
    svdsc_options opt = {0};
    opt.precision = SVDSC_FP64;
    opt.seed = 7;
    svdsc_ctx *ctx = NULL;
    int rc = svdsc_create(&ctx, &A, &opt, NULL);
    if (rc != SVDSC_OK) { printf("create: %s\n", svdsc_strerror(rc)); return 1; }

    svdsc_info info;
    rc = svdsc_solve(ctx, K, 20, 1e-10, 100, NULL, 0, S, U, M, V, N, res, 0, &info);
    if (rc != SVDSC_OK) { printf("solve: %s\n", svdsc_strerror(rc)); return 2; }
    int bad = 0;
    for (int j = 0; j < K; j++) {
        const int i = N - 1 - j;                   /* the largest |d_i| */
        const double want = 1.0 + 0.01 * i;
        if (fabs(S[j] - want) > 1e-12 * want) bad++;
        /* v_j = +-e_{col[i]} (sign rule: its largest entry positive), u_j = e_i d_i / |d_i| */
        if (fabs(V[(size_t)j * N + col[i]] - 1.0) > 1e-10) bad++;
        const double ui = U[(size_t)j * M + i];
        if (fabs(fabs(ui) - 1.0) > 1e-10 || ui * val[i] < 0) bad++;
        if (!(res[j] < 1e-10)) bad++;
        printf("sigma_%d = %.15f (want %.15f) res %.2e\n", j + 1, S[j], want, res[j]);
    }
    printf("restarts %d, products %lld, launches %lld\n", info.restarts, (long long)info.n_matvec,
           (long long)info.n_launches);

    /* error paths: t + 1 > n, bad arguments, a NULL context */
    if (svdsc_solve(ctx, 150, 150, 1e-10, 10, NULL, 0, S, U, M, V, N, res, 0, &info) != SVDSC_ERR_SIZE) bad++;
    if (svdsc_solve(ctx, K, 20, -1.0, 10, NULL, 0, S, U, M, V, N, res, 0, &info) != SVDSC_ERR_ARG) bad++;
    if (svdsc_solve(NULL, K, 20, 1e-10, 10, NULL, 0, S, U, M, V, N, res, 0, &info) != SVDSC_ERR_ARG) bad++;
    if (svdsc_strerror(SVDSC_ERR_SIZE) == NULL) bad++;
    /* the context is still usable after the rejected calls */
    rc = svdsc_solve(ctx, K, 20, 1e-10, 100, NULL, 0, S, U, M, V, N, res, 0, &info);
    if (rc != SVDSC_OK || fabs(S[0] - (1.0 + 0.01 * (N - 1))) > 1e-12) bad++;
    svdsc_destroy(ctx);
    printf("%s (%d problems)\n", bad ? "FAIL" : "OK", bad);
    return bad ? 3 : 0;
}
