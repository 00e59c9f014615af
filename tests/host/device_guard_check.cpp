// Host check of the device verdict behind every GPU entry point's device
// check (csrc/device_guard.h): prints one line per case,
// "ctx_dev cur_dev buf_dev verdict".
#include <cstdio>

#include "device_guard.h"

int main() {
  const int cases[][3] = {
      {0, 0, -1}, {0, 0, 0}, {1, 1, 1}, {1, 1, -1},   // consistent
      {0, 1, -1}, {1, 0, 0}, {0, 1, 1},               // another device is current
      {0, 0, 1}, {1, 1, 0}, {2, 2, 3},                // a buffer on another device
  };
  for (const auto& c : cases)
    std::printf("%d %d %d %d\n", c[0], c[1], c[2], (int)ed::device_verdict(c[0], c[1], c[2]));
  return 0;
}
