/* A C99 client of the library's C ABI: compiles against include/las.h alone and exercises the
 * calls whose argument checks run before any device work (so it runs without a GPU).  Exit
 * status 0 when every check holds; otherwise the number of the first failed check. */
#include <stdio.h>
#include <string.h>

#include "las.h"

#define CHECK(n, cond)                                \
  do {                                                \
    if (!(cond)) {                                    \
      fprintf(stderr, "check %d failed: %s\n", n, #cond); \
      return n;                                       \
    }                                                 \
  } while (0)

int main(void) {
  las_ctx* ctx = (las_ctx*)&ctx;   /* must be reset to NULL by a rejected create */
  double dummy[4] = {0, 0, 0, 0};
  int nact[2] = {2, 2};
  las_dims d;
  int code;

  for (code = LAS_OK; code <= LAS_ERR_UNSUPPORTED; ++code) {
    const char* s = las_status_str((las_status)code);
    CHECK(1, s != NULL && strlen(s) > 0);
  }

  d.nao = 10; d.naux = 20; d.nmo = 10; d.ncore = 2; d.nfrag = 2; d.nact = nact;
  CHECK(2, las_create(NULL, &d, dummy, LAS_FP64, 0, NULL) == LAS_ERR_ARG);
  CHECK(3, las_create(&ctx, NULL, dummy, LAS_FP64, 0, NULL) == LAS_ERR_ARG);
  CHECK(4, las_create(&ctx, &d, NULL, LAS_FP64, 0, NULL) == LAS_ERR_ARG);

  d.nmo = 11;                                       /* nmo > nao */
  CHECK(5, las_create(&ctx, &d, dummy, LAS_FP64, 0, NULL) == LAS_ERR_ARG && ctx == NULL);
  d.nmo = 5;                                        /* ncore + active > nmo */
  CHECK(6, las_create(&ctx, &d, dummy, LAS_SPLIT_BF16, 0, NULL) == LAS_ERR_ARG);
  d.nmo = 10;
  nact[1] = 0;                                      /* an empty fragment */
  CHECK(7, las_create(&ctx, &d, dummy, LAS_FP64, 0, NULL) == LAS_ERR_ARG);
  nact[1] = 2;
  CHECK(8, las_create(&ctx, &d, dummy, (las_precision)3, 0, NULL) == LAS_ERR_ARG);
  d.nmo = 5;                                        /* the packed layout validates the same */
  CHECK(16, LAS_SPLIT_BF16_PACKED == 2 &&
                las_create(&ctx, &d, dummy, LAS_SPLIT_BF16_PACKED, 0, NULL) == LAS_ERR_ARG &&
                ctx == NULL);
  d.nmo = 10;
  d.ncore = 0; d.nfrag = 0;                         /* nothing occupied */
  CHECK(9, las_create(&ctx, &d, dummy, LAS_FP64, 0, NULL) == LAS_ERR_ARG);

  CHECK(10, las_destroy(NULL) == LAS_ERR_ARG);
  CHECK(11, las_sync(NULL) == LAS_ERR_ARG);
  CHECK(12, las_device_bytes(NULL) == 0);
  CHECK(13, las_energy(NULL, dummy, dummy, dummy, dummy, dummy) == LAS_ERR_ARG);
  CHECK(14, las_energy_grad(NULL, dummy, dummy, dummy, dummy, dummy, dummy, NULL) ==
                LAS_ERR_ARG);
  CHECK(15, las_kernel_launches() >= 0);
  printf("ok\n");
  return 0;
}
