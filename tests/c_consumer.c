/*
 * A C99 program that uses the library through include/isg.h alone (no Python, no PyTorch): the
 * 4x4 periodic ferromagnet of Table 1 (Sec. 4) enumerated into a host table, every one of the
 * table's 80 printed cells compared (path of the golden file as argv[1]), the sum and the binomial
 * columns checked, ln Z from isg_thermo compared with Z summed directly over Table 1's cells, and
 * an invalid graph refused with a status and a message. Exit status 0 when everything holds.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "isg.h"

static int fails = 0;
#define CHECK(cond, ...)                        \
    do {                                        \
        if (!(cond)) {                          \
            fprintf(stderr, __VA_ARGS__);       \
            fputc('\n', stderr);                \
            ++fails;                            \
        }                                       \
    } while (0)

int main(int argc, char** argv) {
    if (argc < 2) {
        fprintf(stderr, "usage: %s table1_golden_file\n", argv[0]);
        return 2;
    }
    /* 4x4 periodic square lattice, site (x, y) = 4 x + y, bonds +x and +y, J = 1 */
    int32_t bi[32], bj[32], bJ[32];
    int nb = 0;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
            const int s = 4 * x + y;
            bi[nb] = s; bj[nb] = 4 * ((x + 1) % 4) + y; bJ[nb++] = 1;
            bi[nb] = s; bj[nb] = 4 * x + (y + 1) % 4; bJ[nb++] = 1;
        }
    isg_graph* g = NULL;
    CHECK(isg_graph_create(16, nb, bi, bj, bJ, &g) == ISG_OK, "graph: %s", isg_last_error());
    int32_t e_min = 0, e_step = 0, n_e = 0, m_min = 0, n_m = 0;
    CHECK(isg_graph_bins(g, &e_min, &e_step, &n_e, &m_min, &n_m) == ISG_OK, "bins: %s", isg_last_error());
    CHECK(e_min == -32 && e_step == 2 && n_e == 33 && m_min == -16 && n_m == 17, "geometry %d %d %d %d %d", e_min,
          e_step, n_e, m_min, n_m);
    int64_t* tab = calloc((size_t)n_e * n_m, sizeof(int64_t));
    isg_options opt;
    isg_options_init(&opt);
    CHECK(isg_enumerate(g, NULL, tab, 0, &opt) == ISG_OK, "enumerate: %s", isg_last_error());

    /* Table 1: every printed (Nc, M, E) cell, and no other nonzero bin */
    FILE* f = fopen(argv[1], "r");
    CHECK(f != NULL, "cannot open %s", argv[1]);
    int cells = 0;
    int64_t seen = 0;
    char line[256];
    double Z_cells[3] = {0, 0, 0};
    const double Ts[3] = {1.0, 2.269, 4.0};
    while (f && fgets(line, sizeof line, f)) {
        long long nc;
        int M, E;
        if (line[0] == '#' || sscanf(line, "%lld %d %d", &nc, &M, &E) != 3) continue;
        const int e = (E - e_min) / 2, m = (M - m_min) / 2;
        CHECK(tab[(size_t)e * n_m + m] == nc, "cell E=%d M=%d: %lld, Table 1 %lld", E, M,
              (long long)tab[(size_t)e * n_m + m], nc);
        seen += nc;
        ++cells;
        for (int k = 0; k < 3; ++k) Z_cells[k] += (double)nc * exp(-E / Ts[k]);
    }
    if (f) fclose(f);
    CHECK(cells == 80 && seen == 65536, "Table 1: %d cells, %lld configurations", cells, (long long)seen);
    int64_t total = 0, nonzero = 0;
    for (int i = 0; i < n_e * n_m; ++i) { total += tab[i]; nonzero += tab[i] != 0; }
    CHECK(total == 65536 && nonzero == 80, "sum %lld, %lld nonzero bins", (long long)total, (long long)nonzero);
    for (int m = 0; m < n_m; ++m) {
        int64_t col = 0, binom = 1;
        for (int e = 0; e < n_e; ++e) col += tab[(size_t)e * n_m + m];
        for (int k = 0; k < m; ++k) binom = binom * (16 - k) / (k + 1);
        CHECK(col == binom, "column m=%d: %lld, C(16, m) = %lld", m, (long long)col, (long long)binom);
    }

    /* ln Z on three temperatures at h = 0, host buffers */
    const double h = 0.0;
    double logZ[3], E[3], M[3], C[3], chi[3];
    CHECK(isg_thermo(tab, 0, g, 3, Ts, 1, &h, ISG_FP64, NULL, 0, logZ, E, M, C, chi) == ISG_OK, "thermo: %s",
          isg_last_error());
    for (int k = 0; k < 3; ++k)
        CHECK(fabs(logZ[k] - log(Z_cells[k])) <= 1e-12 * fabs(logZ[k]), "ln Z at T=%g: %.17g vs %.17g", Ts[k], logZ[k],
              log(Z_cells[k]));

    /* an invalid graph: a self-bond */
    int32_t si = 3, sj = 3, sJ = 1;
    isg_graph* bad = NULL;
    CHECK(isg_graph_create(4, 1, &si, &sj, &sJ, &bad) == ISG_ERR_INVALID && bad == NULL, "self-bond accepted");
    CHECK(strlen(isg_last_error()) > 0, "no message for the refused graph");

    free(tab);
    isg_graph_destroy(g);
    if (fails) return 1;
    printf("c consumer ok: Table 1 (80 cells), sum and columns, ln Z at 3 temperatures, refusal\n");
    return 0;
}
