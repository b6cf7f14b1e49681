/*
 * ntt_file.c -- uses the library through its C ABI alone (include/zkntt.h):
 * no Python.  Test helper for tests/test_c_abi.py.
 *
 *   ntt_file check                      host-only checks (no GPU needed)
 *   ntt_file run FIELD LOG_N DIR IN OUT  read 2^LOG_N elements (8 uint32 limbs,
 *                                        Montgomery form) from IN, transform
 *                                        them on the device with
 *                                        zkntt_execute, write OUT; then run the
 *                                        inverse in place and check it returns
 *                                        the input
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "zkntt.h"

static int fail(const char *what, zkntt_status st) {
    fprintf(stderr, "%s: %s\n", what, zkntt_status_str(st));
    return 1;
}

static int host_checks(void) {
    uint32_t mod[8], gen[8];
    int s = 0;
    zkntt_status st = zkntt_field_info(ZKNTT_BLS12_381_FR, mod, gen, &s);
    if (st != ZKNTT_OK) return fail("field_info", st);
    /* r = 0x73eda753...00000001: low limb 1, top limb 0x73eda753, 2-adicity 32 */
    if (mod[0] != 1u || mod[7] != 0x73eda753u || s != 32) {
        fprintf(stderr, "unexpected BLS12-381 constants\n");
        return 1;
    }
    zkntt_plan p = NULL;
    if (zkntt_plan_create(&p, (zkntt_field)7, 10, ZKNTT_FORWARD, NULL) != ZKNTT_EINVAL) {
        fprintf(stderr, "bad field accepted\n");
        return 1;
    }
    if (zkntt_plan_create(&p, ZKNTT_BN254_FR, 29, ZKNTT_FORWARD, NULL) != ZKNTT_EINVAL) {
        fprintf(stderr, "log_n beyond the limit accepted\n");
        return 1;
    }
    if (zkntt_execute(NULL, NULL, NULL, NULL) != ZKNTT_EINVAL) {
        fprintf(stderr, "null plan accepted\n");
        return 1;
    }
    if (zkntt_execute_batch(NULL, NULL, 0, NULL) != ZKNTT_OK) {
        fprintf(stderr, "empty batch rejected\n");
        return 1;
    }
    printf("host checks ok\n");
    return 0;
}

static int run(int field, int log_n, int dir, const char *in_path, const char *out_path) {
    const size_t n = (size_t)1 << log_n, bytes = n * 32;
    uint32_t *h = (uint32_t *)malloc(bytes), *h2 = (uint32_t *)malloc(bytes);
    if (!h || !h2) return 1;
    FILE *f = fopen(in_path, "rb");
    if (!f || fread(h, 1, bytes, f) != bytes) {
        fprintf(stderr, "cannot read %s\n", in_path);
        return 1;
    }
    fclose(f);
    void *d = NULL;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return 1;
    cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
    zkntt_plan fwd = NULL, inv = NULL;
    zkntt_status st = zkntt_plan_create(&fwd, (zkntt_field)field, log_n, (zkntt_dir)dir, NULL);
    if (st != ZKNTT_OK) return fail("plan_create", st);
    st = zkntt_plan_create(&inv, (zkntt_field)field, log_n, (zkntt_dir)(1 - dir), NULL);
    if (st != ZKNTT_OK) return fail("plan_create", st);
    st = zkntt_execute(fwd, d, d, NULL); /* in place, default stream */
    if (st != ZKNTT_OK) return fail("execute", st);
    if (cudaMemcpy(h2, d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    st = zkntt_sync_status(NULL);
    if (st != ZKNTT_OK) return fail("sync_status", st);
    f = fopen(out_path, "wb");
    if (!f || fwrite(h2, 1, bytes, f) != bytes) return 1;
    fclose(f);
    st = zkntt_execute(inv, d, d, NULL);
    if (st != ZKNTT_OK) return fail("execute", st);
    cudaMemcpy(h2, d, bytes, cudaMemcpyDeviceToHost);
    if (memcmp(h, h2, bytes) != 0) {
        fprintf(stderr, "round trip differs\n");
        return 1;
    }
    zkntt_plan_destroy(fwd);
    zkntt_plan_destroy(inv);
    cudaFree(d);
    free(h);
    free(h2);
    printf("run ok\n");
    return 0;
}

int main(int argc, char **argv) {
    if (argc >= 2 && strcmp(argv[1], "check") == 0) return host_checks();
    if (argc == 7 && strcmp(argv[1], "run") == 0)
        return run(atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), argv[5], argv[6]);
    fprintf(stderr, "usage: ntt_file check | run FIELD LOG_N DIR IN OUT\n");
    return 2;
}
