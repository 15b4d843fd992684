/* A plain C client of the library's C ABI (no Python, no C++), for the
 * test of the same name: it checks what a caller can rely on without a
 * GPU -- the header compiles as C, format defaults, packed row sizes,
 * status strings, and argument checks that return before any device work
 * (the device addresses below are never dereferenced).  Exit status 0 when
 * every check holds; each failure is printed. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "vapr.h"

static int fails = 0;
#define CHECK(c)                                                  \
  do {                                                            \
    if (!(c)) {                                                   \
      printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);         \
      ++fails;                                                    \
    }                                                             \
  } while (0)
#define DEV(a) ((void*)(uintptr_t)(a))

int main(void) {
  const vapr_format fp32 = vapr_format_default(8, 23);
  const vapr_format fp16 = vapr_format_default(5, 10);
  const vapr_format e2m1 = vapr_format_default(2, 1);
  const vapr_format e3m2 = vapr_format_default(3, 2);
  const vapr_format bad = {9, 1, 0, 0};
  vapr_format_table t;
  vapr_robot r;

  CHECK(fp16.exp_bits == 5 && fp16.man_bits == 10 && (fp16.flags & VAPR_FMT_IEEE));
  CHECK(vapr_format_supported(fp32) && vapr_format_supported(e2m1) && !vapr_format_supported(bad));
  /* rows padded to 16 bytes; floor(32 / bits) values per 32-bit word */
  CHECK(vapr_packed_row_bytes(156, fp32) == 624);  /* 52 sphere centres */
  CHECK(vapr_packed_row_bytes(156, e2m1) == 80);   /* 8 per word: 20 words */
  CHECK(vapr_packed_row_bytes(7, e3m2) == 16);     /* 5 per word: 2 words */
  CHECK(strlen(vapr_status_string(VAPR_ERR_TOO_LARGE)) > 0);

  t.pos = t.dist = t.grad = t.jgrad = t.xform = fp32;
  memset(&r, 0, sizeof r);
  r.n_joints = 7;
  r.n_spheres = 52;
  r.joint_fixed = (const float*)DEV(256);
  r.sphere_local = (const float*)DEV(512);
  r.sphere_link = (const int32_t*)DEV(768);
  CHECK(vapr_fk(NULL, (const float*)DEV(256), 4, &t, DEV(256), NULL, NULL) == VAPR_ERR_INVALID_ARG);
  CHECK(vapr_fk(&r, (const float*)DEV(256), 0, &t, DEV(256), NULL, NULL) == VAPR_OK);
  CHECK(vapr_fk(&r, (const float*)DEV(256), -1, &t, DEV(256), NULL, NULL) == VAPR_ERR_INVALID_ARG);
  CHECK(vapr_fk(&r, (const float*)DEV(256), 4, &t, DEV(264), NULL, NULL) == VAPR_ERR_MISALIGNED);
  CHECK(vapr_fk(&r, (const float*)DEV(256), VAPR_MAX_CONFIGS + 1, &t, DEV(256), NULL, NULL) ==
        VAPR_ERR_TOO_LARGE);
  t.grad = bad;
  CHECK(vapr_fk(&r, (const float*)DEV(256), 4, &t, DEV(256), NULL, NULL) ==
        VAPR_ERR_UNSUPPORTED_FORMAT);

  if (fails == 0) printf("ok\n");
  return fails != 0;
}
