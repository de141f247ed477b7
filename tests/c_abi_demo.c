/* A plain C caller of libhvp (include/hvp.h): no Python, no PyTorch.
 *
 *   c_abi_demo cpu
 *       calls that need no GPU: hvp_num_gates, hvp_plan_brickwall and the
 *       argument checks of hvp_init; prints one line per check.
 *   c_abi_demo gpu n L Ns in.bin out.bin
 *       in.bin holds, as little-endian doubles, psi_1q (Ns*n*4), U_ref (K*32),
 *       G (K*32) and V (K*32); the program creates a context, runs hvp_hvp
 *       twice and writes loss (1), grad (K*32) and hvp (K*32) to out.bin.
 * Exit status 0 on success; errors print hvp_last_error. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hvp.h"

static int cpu_checks(void) {
    const int K = hvp_num_gates(20, 16);
    printf("num_gates 20 16 = %d\n", K);
    const int P = hvp_plan_brickwall(20, 16, 12, 4, NULL);
    printf("passes 20 16 12 = %d\n", P);
    hvp_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.n = 1;
    cfg.n_layers = 3;
    cfg.n_samples = 2;
    double psi[64] = {0}, ref[512] = {0};
    hvp_ctx *ctx = (hvp_ctx *)0x1;
    const int rc = hvp_init(&ctx, &cfg, psi, ref);
    printf("init n=1 rc = %d ctx_null = %d msg = %s\n", rc, ctx == NULL, hvp_last_error(NULL));
    return (K == 152 && P >= 1 && rc == HVP_EINVAL && ctx == NULL) ? 0 : 1;
}

static int gpu_run(int n, int L, int ns, const char *in_path, const char *out_path) {
    const int K = hvp_num_gates(n, L);
    if (K < 1) return 2;
    const size_t n_psi = (size_t)ns * n * 4, n_g = (size_t)K * 32;
    double *buf = (double *)malloc(sizeof(double) * (n_psi + 3 * n_g));
    double *out = (double *)malloc(sizeof(double) * (1 + 2 * n_g));
    if (!buf || !out) return 3;
    FILE *f = fopen(in_path, "rb");
    if (!f || fread(buf, sizeof(double), n_psi + 3 * n_g, f) != n_psi + 3 * n_g) return 4;
    fclose(f);
    const double *psi = buf, *uref = buf + n_psi, *G = uref + n_g, *V = G + n_g;

    hvp_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.n = n;
    cfg.n_layers = L;
    cfg.n_samples = ns;
    cfg.precision = HVP_C64;
    hvp_ctx *ctx = NULL;
    int rc = hvp_init(&ctx, &cfg, psi, uref);
    if (rc != HVP_OK) {
        fprintf(stderr, "hvp_init: %d %s\n", rc, hvp_last_error(NULL));
        return 5;
    }
    for (int rep = 0; rep < 2 && rc == HVP_OK; ++rep) rc = hvp_hvp(ctx, G, V, out, out + 1, out + 1 + n_g);
    if (rc != HVP_OK) {
        fprintf(stderr, "hvp_hvp: %d %s\n", rc, hvp_last_error(ctx));
        hvp_free(ctx);
        return 6;
    }
    hvp_free(ctx);
    f = fopen(out_path, "wb");
    if (!f || fwrite(out, sizeof(double), 1 + 2 * n_g, f) != 1 + 2 * n_g) return 7;
    fclose(f);
    printf("loss = %.15f\n", out[0]);
    free(buf);
    free(out);
    return 0;
}

int main(int argc, char **argv) {
    if (argc >= 2 && strcmp(argv[1], "cpu") == 0) return cpu_checks();
    if (argc == 7 && strcmp(argv[1], "gpu") == 0)
        return gpu_run(atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), argv[5], argv[6]);
    fprintf(stderr, "usage: c_abi_demo cpu | gpu n L Ns in.bin out.bin\n");
    return 1;
}
