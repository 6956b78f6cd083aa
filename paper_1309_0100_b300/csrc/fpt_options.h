// Frequencies-per-thread options compiled per base size (kept in step with the pgram_p*.cu units).
#pragma once
namespace fredec {
struct FptOptions { int p; int mixed[3]; int nmixed; int fp64[3]; int nfp64; };
static const FptOptions kFptOptions[] = {
    {1, {12, 20, 32}, 3, {2, 4, 0}, 2},
    {3, {8, 12, 20}, 3, {2, 4, 0}, 2},
    {5, {4, 8, 14}, 3, {2, 4, 0}, 2},
    {7, {4, 6, 10}, 3, {1, 2, 4}, 3},
    {9, {3, 5, 8}, 3, {1, 2, 0}, 2},
    {11, {4, 6, 8}, 3, {1, 2, 0}, 2},
    {13, {4, 6, 0}, 2, {1, 0, 0}, 1},
    {15, {2, 3, 0}, 2, {1, 0, 0}, 1},
    {17, {2, 3, 0}, 2, {1, 0, 0}, 1},
    {19, {2, 0, 0}, 1, {1, 0, 0}, 1},
    {21, {2, 0, 0}, 1, {1, 0, 0}, 1},
    {23, {2, 0, 0}, 1, {1, 0, 0}, 1},
    {25, {2, 0, 0}, 1, {1, 0, 0}, 1},
};
}  // namespace fredec
