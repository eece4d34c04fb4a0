// Nested dissection of a regular grid (Sec. 2.2, Alg. 1 specialised to a grid, Sec. 3).
//
// The order I is computed in closed form, one thread per grid node:
//   * a leaf-interior node of leaf box (I,J) goes to 225 * dfs(I,J) + (x%16) + 15 (y%16),
//     where dfs is the depth-first index of the leaf (lower / left child first);
//   * a separator node belongs to the coarsest separator through it.  A vertical line at
//     x is the middle of a depth-(l-1) box whose width is 2^(t+1)-1 with t = ctz(x+1), so
//     its level follows from ctz(x+1) (ctz(y+1) for horizontal lines).  Separators are
//     ordered level L, ..., 1, by depth-first index of the box they cut, then by
//     increasing coordinate along the line.
#include <cstdint>

#include "spalu_internal.h"

namespace spalu {
namespace {

constexpr int MAXL = 64;

struct NDParams {
  int nx, ny, L, nI;
  unsigned long long vcut;     // bit l-1 set when the level-l cut is vertical
  int levelV[32], levelH[32];  // level of a vertical / horizontal line with ctz(coord+1) = t
  int pw[MAXL], ph[MAXL];      // width / height of depth-d boxes, d = 0..L
  int nbits_x[MAXL], nbits_y[MAXL];   // log2 of the tiling at depth d
  long long offset[MAXL];      // first position of the level-l separators in I
  int seplen[MAXL];
};

__device__ int dfs_index(const NDParams& P, int d, int I, int J) {
  int ix = P.nbits_x[d], iy = P.nbits_y[d];
  int v = 0;
  for (int l = 1; l <= d; ++l) {
    int bit;
    if ((P.vcut >> (l - 1)) & 1ull) bit = (I >> (--ix)) & 1;
    else bit = (J >> (--iy)) & 1;
    v = (v << 1) | bit;
  }
  return v;
}

__global__ void nd_perm_kernel(NDParams P, int* perm, int* iperm) {
  long long n = (long long)P.nx * P.ny;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
       g += (long long)gridDim.x * blockDim.x) {
    int x = (int)(g % P.nx), y = (int)(g / P.nx);
    bool vx = ((x + 1) & 15) == 0, hy = ((y + 1) & 15) == 0;
    long long pos;
    if (!vx && !hy) {
      int I = x >> 4, J = y >> 4;
      pos = (long long)NI * dfs_index(P, P.L, I, J) + (x & 15) + LEAF * (y & 15);
    } else {
      int lv = 1 << 30, lh = 1 << 30;
      if (vx) lv = P.levelV[__ffs(x + 1) - 1];
      if (hy) lh = P.levelH[__ffs(y + 1) - 1];
      int l = lv < lh ? lv : lh;
      int d = l - 1;
      int Ip = x / (P.pw[d] + 1), Jp = y / (P.ph[d] + 1);
      int along = (lv < lh) ? (y - Jp * (P.ph[d] + 1)) : (x - Ip * (P.pw[d] + 1));
      pos = P.offset[l] + (long long)dfs_index(P, d, Ip, Jp) * P.seplen[l] + along;
    }
    perm[pos] = (int)g;
    iperm[g] = (int)pos;
  }
}

}  // namespace

void launch_nd_perm(int nx, int ny, int L, const int* vcut_host, int* d_perm, int* d_iperm,
                    cudaStream_t s) {
  NDParams P{};
  P.nx = nx;
  P.ny = ny;
  P.L = L;
  for (int t = 0; t < 32; ++t) P.levelV[t] = P.levelH[t] = 1 << 30;
  int w = nx, h = ny;
  int bxl = 0, byl = 0;
  P.pw[0] = w;
  P.ph[0] = h;
  P.nbits_x[0] = P.nbits_y[0] = 0;
  for (int l = 1; l <= L; ++l) {
    int vc = vcut_host[l];
    if (vc) {
      P.vcut |= 1ull << (l - 1);
      P.seplen[l] = h;
      int t = __builtin_ctz((unsigned)((w + 1) / 2));
      P.levelV[t] = l;
      w = (w - 1) / 2;
      ++bxl;
    } else {
      P.seplen[l] = w;
      int t = __builtin_ctz((unsigned)((h + 1) / 2));
      P.levelH[t] = l;
      h = (h - 1) / 2;
      ++byl;
    }
    P.pw[l] = w;
    P.ph[l] = h;
    P.nbits_x[l] = bxl;
    P.nbits_y[l] = byl;
  }
  long long nleaf = 1ll << L;
  P.nI = (int)(nleaf * NI);
  long long off = P.nI;
  for (int l = L; l >= 1; --l) {
    P.offset[l] = off;
    off += (1ll << (l - 1)) * P.seplen[l];
  }
  long long n = (long long)nx * ny;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  note_launch();
  nd_perm_kernel<<<blocks, 256, 0, s>>>(P, d_perm, d_iperm);
}

}  // namespace spalu
