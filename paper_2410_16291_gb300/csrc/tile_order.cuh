// Ticket-to-tile order of the single-pass builds (host and device, so the
// CPU tests can check the mapping itself).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define SWA_TO_HD __host__ __device__ __forceinline__
#else
#define SWA_TO_HD static inline
#endif

namespace swa {

// The tile (row-major index b*C + s) of ticket k when tickets run along the
// anti-diagonals b + s = d, d = 0, 1, ..., b ascending within a diagonal, on
// a grid of R x C tiles.  Every tile's neighbours above and to the left lie
// one diagonal back, so both look-back chains reach tiles that started about
// one diagonal earlier (in row-major order the left neighbour's ticket is
// the one just before), and every predecessor still has a smaller ticket.
SWA_TO_HD uint32_t diag_tile(uint32_t k, int64_t R, int64_t C)
{
    const int64_t m = R < C ? R : C, M = R < C ? C : R;
    const int64_t T1 = m * (m + 1) / 2, T2 = (M - m) * m;
    auto tri_root = [](int64_t x) {                    // largest e with e(e+1)/2 <= x
        int64_t e = (int64_t)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
        while ((e + 1) * (e + 2) / 2 <= x) ++e;
        while (e > 0 && e * (e + 1) / 2 > x) --e;
        return e;
    };
    int64_t d, j;                                      // diagonal, position along it
    if (k < T1) {                                      // diagonals of length d + 1
        d = tri_root(k);
        j = k - d * (d + 1) / 2;
    } else if (k < T1 + T2) {                          // diagonals of length m
        d = m + (k - T1) / m;
        j = (k - T1) % m;
    } else {                                           // shrinking: count from the end
        const int64_t r = R * C - 1 - k;
        const int64_t e = tri_root(r);                 // diagonal e from the end, length e + 1
        d = R + C - 2 - e;
        j = e - (r - e * (e + 1) / 2);
    }
    const int64_t b = (d - (C - 1) > 0 ? d - (C - 1) : 0) + j;
    return (uint32_t)(b * C + (d - b));
}

}  // namespace swa
