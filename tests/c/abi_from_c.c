/* The C ABI used from plain C99, without a GPU: a 4 x 4 periodic mesh of unit
 * squares, its measures, and the central stencil of cell 0 at order 2, which
 * is enumerated by hand (face neighbours 1, 3, 4, 12, then the diagonals 5 and
 * 7 of the second face layer, the smallest ids at squared distance 2 h^2;
 * Sec. 2.1).  Prints "ok" and exits 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "hfv.h"

#define CHECK(c)                                                       \
    do {                                                               \
        if (!(c)) {                                                    \
            printf("failed: %s (line %d): %s\n", #c, __LINE__, hfv_last_error()); \
            return 1;                                                  \
        }                                                              \
    } while (0)

int main(void)
{
    enum { n = 4 };
    double xyz[(n + 1) * (n + 1) * 2];
    uint8_t type[n * n];
    int64_t ptr[n * n + 1];
    int32_t idx[n * n * 4];
    const double period[2] = {1.0, 1.0};
    for (int j = 0; j <= n; ++j)
        for (int i = 0; i <= n; ++i) {
            xyz[2 * (j * (n + 1) + i)] = (double)i / n;
            xyz[2 * (j * (n + 1) + i) + 1] = (double)j / n;
        }
    ptr[0] = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const int c = j * n + i, v = j * (n + 1) + i;
            type[c] = HFV_QUAD;
            idx[4 * c] = v;
            idx[4 * c + 1] = v + 1;
            idx[4 * c + 2] = v + n + 2;
            idx[4 * c + 3] = v + n + 1;
            ptr[c + 1] = 4 * (c + 1);
        }
    hfv_mesh_desc d;
    d.dim = 2;
    d.n_nodes = (n + 1) * (n + 1);
    d.n_cells = n * n;
    d.node_xyz = xyz;
    d.cell_type = type;
    d.cell_node_ptr = ptr;
    d.cell_node_idx = idx;
    d.period = period;

    hfv_mesh* m = NULL;
    CHECK(hfv_mesh_create(NULL, &m) == HFV_ERR_ARG && strlen(hfv_last_error()) > 0);
    CHECK(hfv_mesh_create(&d, &m) == HFV_OK && m != NULL);
    int64_t nc = 0, nf = 0;
    int dim = 0;
    CHECK(hfv_mesh_info(m, &nc, &nf, &dim) == HFV_OK);
    CHECK(nc == n * n && nf == 2 * n * n && dim == 2);   /* periodic: two faces per cell */

    double vol[n * n], sum = 0.0;
    CHECK(hfv_mesh_volumes(m, vol) == HFV_OK);
    for (int c = 0; c < n * n; ++c) {
        CHECK(fabs(vol[c] - 1.0 / (n * n)) <= 1e-16);
        sum += vol[c];
    }
    CHECK(fabs(sum - 1.0) <= 1e-15);

    int32_t sizes[2] = {0, 0};
    CHECK(hfv_stencils_host(m, 2, sizes, NULL, NULL) == HFV_OK && sizes[0] == 6 && sizes[1] == 6);
    int32_t cen[n * n * 6], dir[n * n * 6 * 6];
    CHECK(hfv_stencils_host(m, 2, sizes, cen, dir) == HFV_OK);
    const int32_t want[6] = {1, 3, 4, 12, 5, 7};
    for (int a = 0; a < 6; ++a) CHECK(cen[a] == want[a]);
    CHECK(hfv_stencils_host(m, 9, sizes, cen, dir) == HFV_ERR_ARG);

    hfv_mesh_destroy(m);
    printf("ok\n");
    return 0;
}
