// Frequencies-per-thread options compiled per base size (generated with the pgram_p*.cu units).
#pragma once
namespace fredec {
struct FptOptions { int p; int mixed[3]; int nmixed; int fp64[3]; int nfp64; };
static const FptOptions kFptOptions[] = {
    {1, {8, 16, 24}, 3, {2, 4, 0}, 2},
    {3, {8, 12, 0}, 2, {2, 4, 0}, 2},
    {5, {6, 10, 0}, 2, {2, 4, 0}, 2},
    {7, {4, 8, 0}, 2, {1, 2, 0}, 2},
    {9, {4, 6, 0}, 2, {1, 2, 0}, 2},
    {11, {4, 6, 0}, 2, {1, 2, 0}, 2},
    {13, {3, 4, 0}, 2, {1, 0, 0}, 1},
    {15, {2, 4, 0}, 2, {1, 0, 0}, 1},
    {17, {2, 3, 0}, 2, {1, 0, 0}, 1},
    {19, {2, 3, 0}, 2, {1, 0, 0}, 1},
    {21, {2, 3, 0}, 2, {1, 0, 0}, 1},
    {23, {2, 0, 0}, 1, {1, 0, 0}, 1},
    {25, {2, 0, 0}, 1, {1, 0, 0}, 1},
};
}  // namespace fredec
