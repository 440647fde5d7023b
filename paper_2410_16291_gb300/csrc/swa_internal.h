// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swa.h"

namespace swa {

constexpr uint64_t kHandleTag = 0x5357414841ULL;   // "SWAHA"
constexpr uint64_t kFreedTag = 0x5357414644ULL;    // "SWAFD"

// Device error word bits (a uint32 in the handle's scratch).
constexpr uint32_t kErrTimeout = 1u;

// Table rows are padded to a multiple of this many elements (256 bytes), so
// that every warp's row segment starts on a full 32-byte sector.
constexpr int64_t kLdAlign = 32;

// Width of the column slice one warp owns in the SAT build: 32 lanes x 8 px.
constexpr int kSliceCols = 256;
constexpr int kPxPerLane = 8;

struct BuildPlan {
    int64_t rows, cols, ld, pitch;
    int dtype;            // SWA_U8 / SWA_U16
    bool with_q;
    bool vec;             // image base and pitch allow 8-pixel vector loads
    int th;               // rows per tile
    int64_t nby, nsx;     // tile bands, column slices
    // scratch layout (byte offsets inside one allocation)
    int64_t off_err, off_cs, off_rs, off_bt, off_stat, off_ticket, scratch_bytes;
    bool twopass;
    bool count;           // table of the indicator "pixel > thr" (S only)
    uint32_t thr;
    bool corner;          // single pass: corner term from corner records (wide images)
    // Corner lattice (single pass with Q): stride (0: none), its size and the
    // caller's arrays for it (S and Q entries at rows and columns one below a
    // multiple of the stride).
    int lat_s;
    int64_t lat_rows, lat_cols, lat_ld;
    uint64_t *lat_S, *lat_Q;
};

struct Handle {
    uint64_t tag;
    int device;
    int64_t rows, cols, ld;
    int dtype;
    uint32_t flags;
    uint64_t *S, *Q;          // device tables (Q may be null)
    uint64_t *LS, *LQ;        // corner lattice of S and Q (null without one)
    int64_t lat_rows, lat_cols, lat_ld;
    int32_t lat_s;            // lattice stride (0: none)
    char *scratch;            // carries, tile status, error word
    int64_t scratch_bytes, table_bytes;
    uint32_t *d_err;          // device error word (inside scratch)
    cudaStream_t stream;      // home stream
    cudaEvent_t use_event;    // joins other streams' calls into the home stream
};

// Memory accounting and the per-device pool.
cudaError_t dev_alloc(void **p, int64_t bytes, cudaStream_t s, swa_status *st);
void dev_free(void *p, int64_t bytes, cudaStream_t s);
void count_launch(int n = 1);

// Brackets one kernel launch with events while profiling is on (see
// swa_profile_begin); counts the launch either way.
class LaunchScope {
  public:
    LaunchScope(const char *name, cudaStream_t s);
    ~LaunchScope();
  private:
    const char *name_;
    cudaStream_t s_;
    int slot_;
};
void set_error(const char *fmt, ...);
uint32_t test_hooks();
// Records the CUDA error; SWA_ENOMEM for allocation failures, else SWA_ECUDA.
swa_status cuda_fail(cudaError_t e, const char *what);
int64_t pixel_bytes(int dtype);
// Overflow guard: every entry of S (and of Q with with_q) of a rows x cols
// image of this dtype is below 2^64 even for an all-maximum image.
bool fits_u64(int64_t rows, int64_t cols, int dtype, bool with_q);

// SAT build (sat_build.cu).  kCountPlan (an internal flag bit): plan the
// table of the indicator "pixel > thr" (staged single pass, S only; the
// caller sets p.thr).
constexpr uint32_t kCountPlan = 1u << 31;
// Single-pass look-back mode for an image nsx column slices wide: edge mode
// with diagonal tickets; with row-major tickets corner records from the
// dtype's threshold on.  The SWA_HOOK_CORNER_MODE test hook forces corner
// mode.
bool corner_mode_for(int64_t nsx, int dtype);
// Ticket order of the single-pass builds: anti-diagonals unless the
// SWA_HOOK_ROW_ORDER test hook is set.
bool ticket_order_diag();
BuildPlan make_plan(int64_t rows, int64_t cols, int64_t pitch, int dtype,
                    uint32_t flags, const void *image);
swa_status launch_build(const BuildPlan &p, const void *image, uint64_t *S,
                        uint64_t *Q, char *scratch, uint32_t *err, cudaStream_t s);

// Window statistics (window_stats.cu).
// One window query: output (i, j) is the window whose top-left pixel is at
// table row row0 + i*sy, column j*sx.  row0 > 0 serves a table that starts
// above the first window (a band of a larger image): corner rows above the
// table's first row read as 0, which is exact when the table starts at or
// above every window's top row.
struct WinDesc {
    int64_t wh, ww, sy, sx, R, C, out_ld;
    int64_t row0;
    uint64_t area;        // window area for the moments (0: wh * ww); a query on a
                          // corner lattice has the lattice's window sides
    uint32_t outputs;
    uint32_t vmax;        // largest pixel value of the table's image (255,
                          // 65535, 1 for a count table; 0: unknown)
    uint64_t *sum;
    double *mean, *std;
};
swa_status launch_windows(const uint64_t *S, const uint64_t *Q, int64_t ld,
                          const WinDesc *w, int n, cudaStream_t s);

}  // namespace swa
