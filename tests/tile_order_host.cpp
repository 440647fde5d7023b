// Host build of the single-pass build's ticket-to-tile mapping, for CPU tests.
#include <stdint.h>
#include <stdlib.h>

#include "tile_order.cuh"

extern "C" {

uint32_t tile_of(uint32_t k, int64_t R, int64_t C) { return swa::diag_tile(k, R, C); }

// 0 if tickets 0 .. R*C-1 map one to one onto the R x C tiles and every
// tile's neighbours above and to the left hold smaller tickets; otherwise
// 1 + the first failing ticket.
int64_t check_grid(int64_t R, int64_t C)
{
    const int64_t n = R * C;
    int64_t *ticket = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int64_t i = 0; i < n; ++i) ticket[i] = -1;
    int64_t bad = 0;
    for (int64_t k = 0; k < n && !bad; ++k) {
        const uint32_t t = swa::diag_tile((uint32_t)k, R, C);
        if ((int64_t)t >= n || ticket[t] >= 0) bad = 1 + k;
        else ticket[t] = k;
    }
    for (int64_t t = 0; t < n && !bad; ++t) {
        const int64_t b = t / C, s = t % C;
        if ((b > 0 && ticket[t - C] >= ticket[t]) || (s > 0 && ticket[t - 1] >= ticket[t]))
            bad = 1 + ticket[t];
    }
    free(ticket);
    return bad;
}
}
