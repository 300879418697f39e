// Constants and plain structs shared by the library's kernels: no runtime API, so that a
// kernel header that needs only these also builds for the host (the test suite's shim).
#pragma once

#include "gsparc.h"

namespace gsparc {

// Footprint cut-off q_max = 2 ln 255: the kernel exp(-q/2) falls to 1/255.
constexpr float kQMax = 11.082527090f;         // 2 * ln(255)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kLog2TMin = -13.287712f;      // log2(1e-4)
constexpr float kDilation = 0.3f;             // px^2 added to diag(Sigma')
constexpr float kRhoFloor = 1e-3f;            // zenith floor on rho, relative to r
constexpr float kDMin = 0.01f;                // metres, floor on the transmitter distance
constexpr double kCLight = 299792458.0;       // m/s
constexpr float kPi = 3.14159265358979f;
constexpr int kTile = GSPARC_TILE;

// A kernel's dynamic shared memory (the test suite's host shim gives it a per-block buffer).
#ifndef GSPARC_DYNAMIC_SMEM
#define GSPARC_DYNAMIC_SMEM(name) extern __shared__ __align__(16) unsigned char name[]
#endif

// First device-detected condition of a call, into the caller's status word (may be null); a
// later condition never overwrites an earlier one.
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(reinterpret_cast<int*>(status), 0, code);
}

// Programmatic dependent launch.  A kernel the host launched with programmatic stream
// serialization (launch_after) may be scheduled while the kernel before it on the stream is still
// running.  grid_dep_wait() returns once that kernel has completed and its writes are visible (at
// once when the launch carried no such dependency), so every such kernel calls it in every block
// before it reads or writes anything the kernels before it touch.  The next kernel is scheduled
// once every block of this grid has exited or called grid_dep_launch(); it still waits in its own
// grid_dep_wait() for this whole grid.  A block that triggers early keeps the dependents' blocks
// resident beside its own remaining work, so only k_tile_count does (its last block's scan is then
// overlapped with the emit pass's footprints); the other kernels let their exit trigger.
#ifdef GSPARC_HOST_SHIM
inline void grid_dep_wait() {}
inline void grid_dep_launch() {}
#else
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

inline int tiles_x(const gsparc_view& v) { return (v.W + kTile - 1) / kTile; }
inline int tiles_y(const gsparc_view& v) { return (v.H + kTile - 1) / kTile; }

// Device-side view constants passed by value to kernels.
struct ViewDev {
    int H, W;
    float rx0, rx1, rx2;
    float V[9];
    float near_dist;
};

}  // namespace gsparc
