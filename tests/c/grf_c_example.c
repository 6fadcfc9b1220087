/*
 * A plain C99 client of the library: only include/grf.h and the CUDA runtime
 * C API, no C++ and no Python.  It shows that the boundary is a C ABI and
 * serves the tests in tests/test_c_abi.py.
 *
 *   grf_c_example host OUT_DIR   draw the modes of one realisation (host
 *                                entry points only) and write them to
 *                                OUT_DIR/modes.bin; check an error path
 *   grf_c_example gpu OUT_DIR    also plan a 40 x 30 grid on the device,
 *                                synthesise Y, K and 2 facies there and
 *                                write Y, K and facies to OUT_DIR
 *
 * Field: Gaussian covariance, sigma^2 = 1.5, mean 0.25, l = (0.15, 0.1),
 * N = 257 modes, seed 99 (Sec. 4.1, Eq. DiscreteFT; Appendix A).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "grf.h"

#define NX 40
#define NY 30
#define NM 257

static int fail(const char *what, int rc) {
    fprintf(stderr, "%s failed: %d (%s)\n", what, rc, grf_last_error());
    return 1;
}

static int write_file(const char *dir, const char *name, const void *p, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof(path), "%s/%s", dir, name);
    FILE *f = fopen(path, "wb");
    if (!f) return 1;
    size_t w = fwrite(p, 1, bytes, f);
    fclose(f);
    return w == bytes ? 0 : 1;
}

int main(int argc, char **argv) {
    if (argc != 3 || (strcmp(argv[1], "host") != 0 && strcmp(argv[1], "gpu") != 0)) {
        fprintf(stderr, "usage: %s host|gpu OUT_DIR\n", argv[0]);
        return 2;
    }
    const int use_gpu = strcmp(argv[1], "gpu") == 0;
    printf("version %s\n", grf_version());

    grf_params p;
    memset(&p, 0, sizeof(p));
    p.family = GRF_GAUSSIAN;
    p.dim = 2;
    p.sigma2 = 1.5;
    p.mean = 0.25;
    p.ell[0] = 0.15;
    p.ell[1] = 0.1;
    p.ell[2] = 1.0;
    p.n_modes = NM;
    p.seed = 99;

    /* an invalid request is refused with a message, nothing else happens */
    grf_params bad = p;
    bad.sigma2 = -1.0;
    static double kappa[NM * 2], rho[NM], psi[NM], a[NM * 2], amp[NM];
    grf_modes m;
    memset(&m, 0, sizeof(m));
    m.n = NM;
    m.dim = 2;
    m.kappa = kappa;
    m.rho = rho;
    m.psi = psi;
    m.a = a;
    m.amp = amp;
    int rc = grf_gen_modes(&bad, &m);
    printf("bad sigma2 -> %d (%s)\n", rc, grf_last_error());
    if (rc != GRF_EINVAL) return 1;

    rc = grf_gen_modes(&p, &m);
    if (rc != GRF_OK) return fail("grf_gen_modes", rc);
    /* modes.bin: a (N x 2), amp (N), psi (N), all double */
    {
        static double buf[NM * 4];
        memcpy(buf, a, sizeof(a));
        memcpy(buf + NM * 2, amp, sizeof(amp));
        memcpy(buf + NM * 3, psi, sizeof(psi));
        if (write_file(argv[2], "modes.bin", buf, sizeof(buf))) return 1;
    }
    const size_t tbytes = grf_table_bytes(NM);
    void *htab = malloc(tbytes);
    if (!htab) return 1;
    rc = grf_pack_table(&m, htab, tbytes);
    if (rc != GRF_OK) return fail("grf_pack_table", rc);
    printf("table %zu bytes\n", tbytes);
    if (!use_gpu) {
        free(htab);
        printf("host ok\n");
        return 0;
    }

    /* cell centres of a 40 x 30 grid of the unit square, x fastest */
    const int n = NX * NY;
    static float hx[NX * NY], hy[NX * NY];
    for (int j = 0; j < NY; ++j)
        for (int i = 0; i < NX; ++i) {
            hx[j * NX + i] = (float)((i + 0.5) / NX);
            hy[j * NX + i] = (float)((j + 0.5) / NY);
        }
    float *dx = NULL, *dy = NULL, *dY = NULL, *dK = NULL;
    uint8_t *dF = NULL;
    void *dplan = NULL, *dtab = NULL, *dws = NULL;
    const int64_t offs[2] = {0, n};
    const size_t pbytes = grf_plan_bytes(n, 1);
    const size_t wbytes = grf_synth_workspace_bytes(n);
    if (cudaMalloc((void **)&dx, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&dy, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&dY, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&dK, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&dF, n) != cudaSuccess || cudaMalloc(&dplan, pbytes) != cudaSuccess ||
        cudaMalloc(&dtab, tbytes) != cudaSuccess || cudaMalloc(&dws, wbytes) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(dx, hx, n * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(dy, hy, n * sizeof(float), cudaMemcpyHostToDevice);
    rc = grf_plan_cells(2, 1, offs, dx, dy, NULL, dplan, pbytes, NULL);
    if (rc != GRF_OK) return fail("grf_plan_cells", rc);
    rc = grf_upload_table(htab, dtab, tbytes, NULL);
    if (rc != GRF_OK) return fail("grf_upload_table", rc);

    grf_map map;
    memset(&map, 0, sizeof(map));
    map.bits = GRF_MAP_Y | GRF_MAP_LOGNORMAL | GRF_MAP_FACIES;
    map.n_thresholds = 1;
    map.thresholds[0] = 0.25f;
    map.k_ref = 1.0f;
    grf_outputs out;
    memset(&out, 0, sizeof(out));
    out.Y = dY;
    out.K = dK;
    out.facies = dF;
    rc = grf_synth_field(dtab, &p, dplan, 0, &map, &out, dws, wbytes, NULL);
    if (rc != GRF_OK) return fail("grf_synth_field", rc);
    int32_t status = -1;
    rc = grf_read_status(dplan, &status, NULL);
    if (rc != GRF_OK || status != 0) return fail("grf_read_status", rc ? rc : status);

    static float hY[NX * NY], hK[NX * NY];
    static uint8_t hF[NX * NY];
    cudaMemcpy(hY, dY, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(hK, dK, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (cudaMemcpy(hF, dF, n, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    if (write_file(argv[2], "Y.bin", hY, sizeof(hY)) || write_file(argv[2], "K.bin", hK, sizeof(hK)) ||
        write_file(argv[2], "facies.bin", hF, sizeof(hF)))
        return 1;
    grf_release(dplan);
    cudaFree(dx);
    cudaFree(dy);
    cudaFree(dY);
    cudaFree(dK);
    cudaFree(dF);
    cudaFree(dplan);
    cudaFree(dtab);
    cudaFree(dws);
    free(htab);
    printf("gpu ok\n");
    return 0;
}
