// Discrete velocity sets of the two-lattice free energy LBM (Sec. 2.2,
// Fig. discVeloSets: D2Q9 and D3Q19).  The paper prints no table; the
// weights are the textbook ones (w = 4/9, 1/9, 1/36 and 1/3, 1/18, 1/36,
// cs^2 = 1/3).  The direction order is the canonical exchange order of the C
// ABI (include/fre.h).  Everything is a constexpr function of the direction
// index so that fully unrolled loops fold the velocities into immediates.
#pragma once

namespace fre {

template <int Q>
struct Lat;

template <>
struct Lat<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // opposite direction: 1<->3, 2<->4, 5<->7, 6<->8
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i < 5 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
    }
};

template <>
struct Lat<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 13 || i == 15) ? 1
             : ((i == 2 || i == 8 || i == 10 || i == 14 || i == 16) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 7 || i == 11 || i == 14 || i == 17) ? 1
             : ((i == 4 || i == 8 || i == 12 || i == 13 || i == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 9 || i == 11 || i == 16 || i == 18) ? 1
             : ((i == 6 || i == 10 || i == 12 || i == 15 || i == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    // opposite pairs are (1,2), (3,4), ..., (17,18)
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

}  // namespace fre
