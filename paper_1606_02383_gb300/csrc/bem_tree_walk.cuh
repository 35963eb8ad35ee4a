// bem_tree_walk.cuh -- the per-point walk of the source octree behind the
// off-surface evaluation (the field at points in the fluid, Section 2.5,
// through the FMM of Section 2.3).
//
// A field point x lies in the box t of the finest level L (integer
// coordinates, extended beyond the root cube: a point outside it gets
// coordinates below 0 or at and above 2^L).  Every source box D of level l
// is taken in one of three ways:
//   far   D does not touch the point's box at level l (t >> (L - l)), and the
//         gap between the point's level-L box and D is at least 4 h_max(D),
//         so no element of D needs the near-singular rule at x: the multipole
//         of D is evaluated at x (M2P).  (WalkTree.gap_scale2 scales the
//         squared gap: the vertex gradient, regular rule only, asks for one
//         h_max);
//   near  otherwise, if D is a leaf: its elements are summed directly, each
//         with the rule its distance calls for;
//   open  otherwise: D's children are walked.
// The walk starts from every box of level 2.  Every source element is
// therefore counted exactly once, in the multipole of one far box or in one
// near leaf.  The multipole converges at x: x is at least 1.5 w_l from D's
// centre in the max norm while D's sources are within (sqrt 3 / 2) w_l of it.
#pragma once
#include "bem_common.cuh"

struct WalkLevel {
  const int* coord = nullptr;              // [nbox][3]
  const unsigned char* internal = nullptr;  // [nbox]
  const int* child0 = nullptr;              // [nbox]
  const int* nchild = nullptr;              // [nbox]
  const float* gap2 = nullptr;              // [nbox] (4 h_max / w_L)^2: the smallest squared gap, in level-L widths
  const double* centre = nullptr;           // [nbox][3]
  const int* start = nullptr;               // [nbox] first element (sorted order)
  const int* end = nullptr;                 // [nbox]
  int nbox = 0;
};

struct WalkTree {
  WalkLevel lv[BEM_MAXLEV + 1];
  int L = 0;
  double lo[3] = {0, 0, 0};  // corner of the root cube
  double wL = 0;             // width of a level-L box
  float gap_scale2 = 1.0f;   // the far test's gap in units of 4 h_max(D), squared
};

// Field points in walk order (bem_eval_fmm.cu): sorted along a Morton curve of
// their level-L boxes.  perm[i] is the caller's index of walk point i, spts and
// tcs its coordinates and box; nearflag / near_list / n_near the points whose
// walk has near leaves, filled by the far pass and bem_walk_near_list.
struct WalkOrder {
  unsigned long long *keys_in = nullptr, *keys = nullptr;
  int *idx_in = nullptr, *perm = nullptr, *tcs = nullptr, *nearflag = nullptr, *near_list = nullptr,
      *n_near = nullptr;
  double* spts = nullptr;
  void *tmp = nullptr, *tmp2 = nullptr;
};
WalkTree bem_walk_tree(const bem_handle* h);
// allocates wo's arrays (stream-ordered) and sorts the np points; on failure
// the arrays allocated so far stay in wo for bem_walk_free
int bem_walk_order(const WalkTree& wt, int64_t np, const double* points, WalkOrder& wo, cudaStream_t s);
int bem_walk_near_list(int64_t np, WalkOrder& wo, cudaStream_t s);
void bem_walk_free(WalkOrder& wo, cudaStream_t s);

// stack bound: one level-2 box, then at most 7 pending siblings on each of
// the levels 3 .. 10 and the 8 children of the box being opened
#define WALK_STACK 72
#define WALK_COORD_MAX (1 << 20)
// far boxes a lane of a walking team lists before it evaluates them
#define WALK_OWN 48

// the level-L box of a point (clamped far outside: such a point stays far
// from every box)
__device__ __forceinline__ void walk_box_of(const WalkTree& wt, const double* x, int* t) {
  for (int a = 0; a < 3; ++a) {
    double c = floor((x[a] - wt.lo[a]) / wt.wL);
    c = fmin(fmax(c, -(double)WALK_COORD_MAX), (double)WALK_COORD_MAX);
    t[a] = (int)c;
  }
}

// visit(kind, level, box): kind 0 = far (M2P), 1 = near leaf (direct sum)
template <typename Visit>
__device__ __forceinline__ void tree_walk(const WalkTree& wt, const int* t, Visit&& visit) {
  int stack[WALK_STACK];
  const int nb2 = wt.lv[2].nbox;
  for (int b2 = 0; b2 < nb2; ++b2) {
    int sp = 0;
    stack[sp++] = (2 << 24) | b2;
    while (sp > 0) {
      const int code = stack[--sp];
      const int l = code >> 24, b = code & 0xFFFFFF;
      const WalkLevel& lv = wt.lv[l];
      const int sh = wt.L - l;
      bool adj = true;
      long long g2 = 0;
      for (int a = 0; a < 3; ++a) {
        const int d = lv.coord[3 * b + a];
        const int ta = t[a] >> sh;  // arithmetic shift: floor for negative coordinates
        if (d - ta > 1 || ta - d > 1) adj = false;
        const long long lo = (long long)d << sh, hi = lo + (1LL << sh);
        long long g = 0;
        if (lo - t[a] - 1 > g) g = lo - t[a] - 1;
        if (t[a] - hi > g) g = t[a] - hi;
        g2 += g * g;
      }
      if (!adj && (float)g2 >= wt.gap_scale2 * lv.gap2[b]) {
        visit(0, l, b);
        continue;
      }
      if (!lv.internal[b]) {
        visit(1, l, b);
        continue;
      }
      const int c0 = lv.child0[b], nc = lv.nchild[b];
      for (int c = 0; c < nc; ++c) stack[sp++] = ((l + 1) << 24) | (c0 + c);
    }
  }
}

// the walk's view of a handle's tree (host side)
WalkTree bem_walk_tree(const bem_handle* h);
