// kd_persist.h -- the persistent batch kernel's plan (kd_persist.cu), shared with the host
// API (kd_api.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include "kd_internal.h"

namespace kd {

// One member of a persistent batch launch: its sweeps' arguments (the y sweep with the
// kinetic factor; the x sweep with the potential factor for tau = dt, and for tau = dt/2
// as the closing half sweep; the step index is set per item), log2 grid sizes, and work
// items per sweep.
// 16-byte aligned with a size that is a multiple of 16, so that every member of the
// device array, and each of its SweepArgs, starts on a 16-byte boundary (the kernel copies
// them to shared memory in 16-byte words)
struct alignas(16) PersistMember {
    SweepArgs y, x, xc;
    int lx, ly;
    int iy, ix;      // work items per y / x sweep
    int cy, cx;      // CTA-fulls of blocks per y / x sweep
    int gy, gx;      // CTA-fulls per work item (the last item may hold fewer)
    int vy_alt, vx_alt;   // 1: the axis runs the second of the kernel's two launch variants
    int* status;
};
static_assert(sizeof(SweepArgs) % 16 == 0, "SweepArgs is copied in 16-byte words");
static_assert(sizeof(PersistMember) % 16 == 0 && alignof(PersistMember) == 16,
              "persistent members start on 16-byte boundaries");

struct PersistPlan {
    const PersistMember* members;
    int n;
    const int* pre_y;        // [n + 1] prefix sums of the members' y items
    const int* pre_x;        // [n + 1] prefix sums of the members' x items
    int y_items, items_per_step;
    int chunk;               // steps in this launch
    int closing;             // the chunk's last x sweep is the closing half sweep
    unsigned* next;          // work queue head (zero before the launch)
    unsigned* done;          // [n] completed items per member (zero before the launch)
    int* abort;              // set when a bounded wait gives up (zero before the launch)
    long long budget_cycles; // bound of one dependency wait
    int hold_item;           // test hook: this item's completion is never signalled (-1: none)
};

// Axes of 2^logn points the persistent kernel holds (16 ... 512).
bool persist_supported(int logn);
// CTA-fulls of blocks of one sweep over `lines` lines of 2^logn points (axis AXIS_X or
// AXIS_Y, launch variant alt 0/1 of the axis); a work item runs one or more of them.
int persist_ctas(int axis, int alt, int logn, int lines);
// The persistent kernel holds two launch variants per axis of 2^logn points (v0 the
// default, v1 the other; v1 = v0 where only one fits its CTA); persist_variant_alt gives 1
// for a simulation's variant that is v1, else 0 (the member then runs v0).
void persist_variants(int axis, int logn, int* v0, int* v1);
int persist_variant_alt(int axis, int variant, int logn);
cudaError_t launch_persist(const PersistPlan& p, cudaStream_t s);

}  // namespace kd
