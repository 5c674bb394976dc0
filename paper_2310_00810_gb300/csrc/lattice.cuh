// Lattice tables for the device code: D2Q9 and D3Q19 velocity sets,
// weights and opposite directions (section 2.1 of arXiv 2310.00810, Fig. 1).
// Every accessor is constexpr so that fully unrolled loops fold the tables
// into immediates.
#pragma once

#include <cstdint>

namespace lbm {

template <int Q>
struct Lattice;

// D2Q9: rest, E, N, W, S, NE, NW, SW, SE (the order of Fig. 1 / Eq. 18).
template <>
struct Lattice<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

// D3Q19: rest, six axis links, twelve edge links; opposite pairs adjacent.
template <>
struct Lattice<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

constexpr uint32_t kLinkSolid = 0x80000000u;

}  // namespace lbm
