/* A plain C99 caller of the C ABI (no CUDA headers, no torch): the host-only
 * entry points -- status names, the LJ pair table, the workspace plan and the
 * Appendix buffer estimate -- print their results for the test to compare. */
#include <stdio.h>

#include "nbcluster.h"

int main(void) {
    const double sigma[2] = {0.3166, 0.0}, eps[2] = {0.650, 0.0};
    float c6c12[2 * 2 * 2];
    nb_status s = nb_lj_combine(2, sigma, eps, NB_COMB_LB, c6c12);
    printf("lj %d %.9e %.9e\n", s, (double)c6c12[0], (double)c6c12[1]);

    const int n = 24000;
    const double box[3] = {6.21, 6.21, 6.21};
    size_t bytes = 0;
    s = nb_workspace_bytes(8, 1, &n, box, 1.1, 2, 0.0, &bytes);
    printf("plan %d %zu\n", s, bytes);
    const int big = 1100000000;
    const double dilute[3] = {2802.04, 2802.04, 2802.04};
    s = nb_workspace_bytes(8, 1, &big, dilute, 1.1, 2, 0.0, &bytes);
    printf("refused %d %s\n", s, nb_status_string(s));

    /* 8,000 water molecules in 6.21 nm: O (LJ type 0) and H (type 1) */
    const nb_particle_class cls[2] = {{8000.0, 15.9994, -0.82, 0}, {16000.0, 1.008, 0.41, 1}};
    nb_params p = {NB_ELEC_EWALD, 0, 1.0f, 0.0f, 3.12f};
    double drift = 0.0, rb = 0.0;
    s = nb_buffer_drift(2, cls, 2, c6c12, 6.21 * 6.21 * 6.21, &p, 0.1, 0.038, 300.0, &drift);
    printf("drift %d %.12e\n", s, drift);
    s = nb_buffer_size(2, cls, 2, c6c12, 6.21 * 6.21 * 6.21, &p, 0.038, 300.0, 0.00249, &rb);
    printf("size %d %.9f\n", s, rb);

    /* the frame runner without a context: refused before any CUDA call */
    nb_frames fr = {0};
    fr.n_frames = 1;
    s = nb_run_frames(NULL, &p, &fr, NULL, NULL);
    printf("frames %d %s\n", s, nb_status_string(s));
    return 0;
}
