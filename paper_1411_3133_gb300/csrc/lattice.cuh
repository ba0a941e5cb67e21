// D3Q41 velocity set (Table I) in the library's pair order.
//
// Index 0 is the rest velocity; for k = 0..19 the indices 2k+1 and 2k+2 hold
// a velocity c and its opposite -c. Pairs are grouped by Table I's shells:
// |c| = 1 along an axis (3 pairs), (+-1,+-1,0)-type (6), (+-1,+-1,+-1) (4),
// +-3 along an axis (3), (+-3,+-3,+-3) (4). The weights are Table I's
// closed forms; cs^2 = 1 - sqrt(2/5) = 1 - sqrt(10)/5 (Sec. II).
#pragma once

namespace lbgm {

constexpr int Q = 41;
constexpr int NPAIR = 20;

// sqrt(10) to double precision; checked against std::sqrt at context creation.
constexpr double SQRT10 = 3.16227766016837933199889354443271853;
constexpr double CS2 = 1.0 - SQRT10 / 5.0;

constexpr double W_REST = 2.0 / 2025.0 * (5045.0 - 1507.0 * SQRT10);
constexpr double W_AX1 = 37.0 / (5.0 * SQRT10) - 91.0 / 40.0;
constexpr double W_FACE1 = (55.0 - 17.0 * SQRT10) / 50.0;
constexpr double W_BODY1 = (233.0 * SQRT10 - 730.0) / 1600.0;
constexpr double W_AX3 = (295.0 - 92.0 * SQRT10) / 16200.0;
constexpr double W_BODY3 = (130.0 - 41.0 * SQRT10) / 129600.0;

// representative (first) velocity of each pair, and its weight
struct PairDef {
  int x, y, z;
  double w;
};

constexpr PairDef PAIRS[NPAIR] = {
    {1, 0, 0, W_AX1},    {0, 1, 0, W_AX1},    {0, 0, 1, W_AX1},
    {1, 1, 0, W_FACE1},  {1, -1, 0, W_FACE1}, {1, 0, 1, W_FACE1},
    {1, 0, -1, W_FACE1}, {0, 1, 1, W_FACE1},  {0, 1, -1, W_FACE1},
    {1, 1, 1, W_BODY1},  {1, 1, -1, W_BODY1}, {1, -1, 1, W_BODY1},
    {1, -1, -1, W_BODY1},
    {3, 0, 0, W_AX3},    {0, 3, 0, W_AX3},    {0, 0, 3, W_AX3},
    {3, 3, 3, W_BODY3},  {3, 3, -3, W_BODY3}, {3, -3, 3, W_BODY3},
    {3, -3, -3, W_BODY3},
};

// Host-side helpers: velocity component and weight of population l (0..40).
constexpr int vel(int l, int axis) {
  return l == 0 ? 0
                : ((l - 1) % 2 == 0 ? 1 : -1) *
                      (axis == 0 ? PAIRS[(l - 1) / 2].x
                                 : axis == 1 ? PAIRS[(l - 1) / 2].y : PAIRS[(l - 1) / 2].z);
}
constexpr double weight(int l) {
  return l == 0 ? W_REST : PAIRS[(l - 1) / 2].w;
}
constexpr int opposite(int l) {
  return l == 0 ? 0 : ((l - 1) % 2 == 0 ? l + 1 : l - 1);
}

}  // namespace lbgm
