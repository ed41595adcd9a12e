// serve_internal.h -- layout shared by the serving scheduler (serve.cpp) and the
// persistent serving kernel (serve.cu).  Not part of the public ABI.
#pragma once

#include "dqj_internal.h"

namespace dqj {

constexpr int kMaxSlots = 64;        // requests resident on the device at once
constexpr int DQJ_NSTATS_DEV = 10;   // = DQJ_NSTATS

enum : unsigned { kPhaseMarch = 0, kPhaseBisect = 1, kPhaseDone = 2 };

// One resident request.  Words that warps update are generation-tagged: the high
// 32 bits hold the request's generation (the low 32 bits of seq).
struct alignas(16) ServeSlot {
    unsigned long long seq;         // admission sequence; 0 while empty or being rewritten
    unsigned long long phase;       // (gen << 32) | kPhase*
    unsigned long long tile_claim;  // (gen << 32) | next march tile
    unsigned long long tile_done;   // (gen << 32) | march tiles completed
    unsigned long long hit_claim;   // (gen << 32) | next hit-list entry
    unsigned long long hit_done;    // (gen << 32) | hit-list entries completed
    unsigned ntiles;                // march tiles of the frame
    unsigned hit_total;             // hit-list length, set when the march completes
    unsigned pad[2];
    Scratch sc;                     // the request's counters and hit list
    FrameDesc fd;                   // frame constants and caller's output planes
};
static_assert(sizeof(Scratch) % 16 == 0, "Scratch is copied as uint4");
static_assert(sizeof(FrameDesc) % 16 == 0, "FrameDesc is copied as uint4");

struct ServeCtl {
    ServeSlot *slots;               // device array of kMaxSlots
    unsigned *done_flags;           // mapped host memory: generation of the last finished request per slot
    unsigned *stop;                 // mapped host memory: non-zero asks the kernel to exit
    unsigned long long idle_ns;     // a warp with no work for this long exits
};

cudaError_t serve_launch(const ServeCtl &ctl, int num_sms, cudaStream_t st);

}  // namespace dqj
