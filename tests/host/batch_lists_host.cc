// The batch's work lists on the host: for a set of grids, every list kind and every block
// shape the batch launches it with, the layout hweno_batch_init builds (batch_layout)
// read through the kernels' own item decoding (find_case, then tile_pos for the
// per-cell kernels, or the tile kernels' (bx, by) split of a case's items) must cover
// each position of each case's launch region exactly once.  Arguments: nx ny pairs.
// Output: one line per (kind, shape): kind bx by total bad, where bad counts the
// positions covered other than once plus the decoded positions of the wrong case.
#include "shim.h"
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "hweno_batch.cuh"

namespace hw {
double cons_smem[CONS_SMEM_BYTES / sizeof(double)];  // the dynamic shared memory the bodies name
double dr_smem[DR_SMEM_BYTES / sizeof(double)];
}  // namespace hw

using namespace hw;

int main(int argc, char** argv) {
  if (argc < 3 || (argc - 1) % 2) return 1;
  const int n = (argc - 1) / 2;
  std::vector<Grid> grids(n);
  for (int c = 0; c < n; c++) {
    hweno_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.nx = atoi(argv[1 + 2 * c]);
    cfg.ny = atoi(argv[2 + 2 * c]);
    cfg.x1 = 1.0; cfg.y1 = 1.0; cfg.gamma = 1.4; cfg.Pr = 0.72; cfg.Re = 100.0;
    grids[c] = make_grid(cfg);
  }
  auto grid_of = [&](int c) -> const Grid& { return grids[c]; };
  const int tuned[4][2] = {{32, 4}, {16, 8}, {64, 2}, {128, 1}};
  for (int k = 0; k < BR_N; k++) {
    std::vector<std::pair<int, int>> shapes;
    if (k <= BR_INT)
      for (auto& s : tuned) shapes.push_back({s[0], s[1]});
    if (k == BR_GRAD) shapes.push_back({32, DR_THREADS / 32});  // kb_dr
    if (k == BR_GHOST || k == BR_SPLIT) shapes.push_back({128, 1});
    if (k == BR_FR || k == BR_FRA) shapes.push_back({FR_TX, FR_TY});
    if (k == BR_GT) shapes.push_back({GT_X, GT_Y});
    for (auto [bx, by] : shapes) {
      std::vector<int> lay(3 * n + 1);
      const int total = batch_layout(k, n, grid_of, bx, by, lay.data());
      const TileList L{lay.data(), lay.data() + (n + 1), lay.data() + (2 * n + 1)};
      std::vector<std::vector<unsigned char>> cnt(n);
      std::vector<int> wx(n), wy(n), wz(n);
      for (int c = 0; c < n; c++) {
        batch_region(k, grids[c], wx[c], wy[c], wz[c]);
        cnt[c].assign((size_t)wx[c] * wy[c] * wz[c], 0);
      }
      long long bad = 0;
      const bool tiles = k == BR_FR || k == BR_FRA || k == BR_GT;
      for (int t = 0; t < total; t++) {
        const int c = find_case(L.start, n, t);
        if (c < 0 || c >= n || t < L.start[c] || t >= L.start[c + 1]) {
          bad++;
          continue;
        }
        blockDim = {(unsigned)bx, (unsigned)by, 1};
        for (int ty = 0; ty < by; ty++)
          for (int tx = 0; tx < bx; tx++) {
            threadIdx = {(unsigned)tx, (unsigned)ty, 0};
            int gx, gy, gz = 0;
            if (tiles) {  // the tile kernels: item l of the case is tile (l mod tx, l div tx)
              const int l = t - L.start[c];
              const int tby = l / L.tx[c], tbx = l - tby * L.tx[c];
              gx = tbx * bx + tx;
              gy = tby * by + ty;
            } else {
              tile_pos(L, c, t, gx, gy, gz);
            }
            if (gz < 0 || gz >= wz[c]) {
              bad++;
              continue;
            }
            if (gx < wx[c] && gy < wy[c]) cnt[c][((size_t)gz * wy[c] + gy) * wx[c] + gx]++;
          }
      }
      for (int c = 0; c < n; c++)
        for (unsigned char v : cnt[c]) bad += v != 1;
      printf("%d %d %d %d %lld\n", k, bx, by, total, bad);
    }
  }
  return 0;
}
