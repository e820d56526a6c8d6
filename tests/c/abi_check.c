/* Compiled as C11 against include/prtgs.h and linked with libprtgs.so by tests/test_c_header.py:
 * the header is plain C, and the host-side entry points answer without a GPU (version,
 * error strings, workspace sizes, argument validation). Prints "ok" and exits 0 on success. */
#include <stdio.h>
#include <string.h>

#include "prtgs.h"

#define CHECK(cond)                                          \
  do {                                                       \
    if (!(cond)) {                                           \
      fprintf(stderr, "check failed line %d: %s\n", __LINE__, #cond); \
      return 1;                                              \
    }                                                        \
  } while (0)

int main(void) {
  CHECK(prtgs_version() >= 10000);
  CHECK(strncmp(prtgs_strerror(PRTGS_ERR_WORKSPACE), "workspace", 9) == 0);
  prtgs_transfer_params p;
  memset(&p, 0, sizeof p);
  p.sh_order = 3;
  p.n_dirs = 256;
  p.flags = PRTGS_SHADOW | PRTGS_BOUNCE;
  p.n_bounces = 2;
  CHECK(prtgs_transfer_workspace_size(100000, 0, &p) > 0);
  CHECK(prtgs_build_bvh_workspace_size(1000, 1) > 0);
  CHECK(prtgs_render_relit_workspace_size(1000, 3, 64, 48, 1 << 16) > 0);
  /* null arguments are refused before any device work */
  prtgs_gaussians g;
  memset(&g, 0, sizeof g);
  g.n = 10;
  prtgs_bvh bvh;
  memset(&bvh, 0, sizeof bvh);
  CHECK(prtgs_build_bvh(&g, &bvh, NULL, NULL, 0, NULL) == PRTGS_ERR_INVALID_ARG);
  CHECK(prtgs_precompute_transfer(&g, NULL, &p, NULL, NULL, NULL, NULL, 0, NULL, NULL, 0, NULL) ==
        PRTGS_ERR_INVALID_ARG);
  /* struct layouts, compared with the binding's mirrors by the Python side */
  printf("sizes %zu %zu %zu %zu %zu %zu %zu\n", sizeof(prtgs_gaussians), sizeof(prtgs_bvh),
         sizeof(prtgs_transfer_params), sizeof(prtgs_camera), sizeof(prtgs_render_state), sizeof(prtgs_tune_transfer),
         sizeof(prtgs_tune_relight));
  printf("ok\n");
  return 0;
}
