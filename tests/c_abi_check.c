/* A plain C99 program against include/hp.h and libhp.so, with no Python and
 * no torch: builds the 32-stage stencil chain, fuses it four stages per group,
 * and queries the lowering and the bounds inference (host-only calls, no GPU
 * needed).  Built and run by tests/test_c_abi.py; prints "ok" on success. */
#include <stdio.h>
#include <string.h>

#include "hp.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    hp_status s_ = (call);                                                   \
    if (s_ != HP_OK) {                                                       \
      printf("FAIL %s: status %d: %s\n", #call, (int)s_, hp_last_error());  \
      return 1;                                                              \
    }                                                                        \
  } while (0)

int main(void) {
  const float binomial[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
  const float box[5] = {0.2f, 0.2f, 0.2f, 0.2f, 0.2f};
  const int in_dtype = HP_F32, in_channels = 1;
  hp_pipeline* p = NULL;
  CHECK(hp_pipeline_create(&p, 1, &in_dtype, &in_channels));
  int prev = -1, id = -1;
  for (int k = 0; k < 32; ++k) {
    hp_stage_desc d;
    memset(&d, 0, sizeof d);
    d.kind = HP_STENCIL;
    d.n_inputs = 1;
    d.inputs = &prev;
    d.rx = d.ry = 2;
    d.wx = d.wy = (k % 2 == 0) ? binomial : box;
    d.storage = HP_F32;
    d.channels = 1;
    CHECK(hp_add_stage(p, &d, &id));
    if (id != k) {
      printf("FAIL: stage id %d, expected %d\n", id, k);
      return 1;
    }
    prev = id;
  }
  CHECK(hp_set_output(p, id));

  int groups[32], tw[8], th[8], thr[8], sy[8];
  for (int k = 0; k < 32; ++k) groups[k] = k / 4;
  for (int g = 0; g < 8; ++g) {
    tw[g] = 64;
    th[g] = 64;
    thr[g] = 256;
    sy[g] = 8;
  }
  hp_schedule sc = {32, groups, 8, tw, th, thr, sy, NULL};
  CHECK(hp_schedule_set(p, &sc));
  int n = 0;
  CHECK(hp_group_count(p, &n));
  const int W = 2560, H = 1536;
  hp_group_info info;
  CHECK(hp_group_info_get(p, &W, &H, 0, &info));
  if (n != 8 || info.kernel != HP_KERNEL_STENCIL_CHAIN || info.n_members != 4 || info.grid_x != 40 ||
      info.grid_y != 24 || info.threads != 256) {
    printf("FAIL: groups %d kernel %d members %d grid %dx%d threads %d\n", n, info.kernel, info.n_members,
           info.grid_x, info.grid_y, info.threads);
    return 1;
  }
  /* group 1 (stages 4..7) for the output tile [64, 128) x [64, 128): stage 4 is
   * needed 2 px wider per remaining stage on every side */
  int rects[4 * 32];
  CHECK(hp_infer_bounds(p, &W, &H, 1, 64, 64, 64, 64, rects, 32));
  const int* r4 = rects + 4 * 4;
  const int* r7 = rects + 4 * 7;
  if (r7[0] != 64 || r7[1] != 64 || r7[2] != 128 || r7[3] != 128 || r4[0] != 58 || r4[1] != 58 || r4[2] != 134 ||
      r4[3] != 134) {
    printf("FAIL: bounds (%d %d %d %d) (%d %d %d %d)\n", r7[0], r7[1], r7[2], r7[3], r4[0], r4[1], r4[2], r4[3]);
    return 1;
  }
  /* an invalid call returns a status and a message, never aborts */
  if (hp_set_output(p, 99) == HP_OK || hp_last_error()[0] == '\0') {
    printf("FAIL: bad output id accepted\n");
    return 1;
  }
  CHECK(hp_pipeline_destroy(p));
  printf("ok\n");
  return 0;
}
