// serve_internal.h -- layout shared by the serving scheduler (serve.cpp) and the
// persistent serving kernel (serve.cu).  Not part of the public ABI.
#pragma once

#include "dqj_internal.h"

namespace dqj {

constexpr int kMaxSlots = 64;        // requests resident on the device at once
constexpr int kReqBlocks = 1024;     // request control blocks (see ReqBlock)
constexpr int DQJ_NSTATS_DEV = 10;   // = DQJ_NSTATS

// A request's phases, in order.  FP32 + FP64 recheck requests pass through
// kPhaseRecheck (FP64 recheck of the queued samples) and kPhaseFixup (FP64
// re-render of the pixels whose FP64 escape count differed); each phase is
// skipped when it has no work.
enum : unsigned { kPhaseMarch = 0, kPhaseBisect = 1, kPhaseRecheck = 2, kPhaseFixup = 3, kPhaseDone = 4 };

// Control block of one admitted request.  Written by the host before the
// request is published and, apart from its counters, never changed afterwards.
// The host hands a block to a new request only after every warp of the launch
// that could have seen its previous request has exited, so a warp holding a
// stale view finds only exhausted claim counters and can do no harm.
struct alignas(128) ReqBlock {
    unsigned long long tile_claim;  // next march tile (claims may run past ntiles)
    unsigned long long tile_done;   // march tiles completed
    unsigned long long hit_claim;   // next hit-list entry
    unsigned long long hit_done;    // hit-list entries completed
    unsigned phase;                 // kPhase*
    unsigned ntiles;                // march tiles of the frame
    unsigned hit_total;             // hit-list length, set when the march completes
    unsigned slot;                  // slot the request occupies
    unsigned gen;                   // generation reported through the slot's done flag
    unsigned recheck;               // 1: FP32 + FP64 recheck request
    unsigned q_total;               // recheck-queue length, set when the bisection completes
    unsigned f_total;               // re-render list length, set when the recheck completes
    unsigned long long q_claim, q_done;  // recheck queue entries claimed / completed
    unsigned long long f_claim, f_done;  // re-rendered pixels claimed / completed
    Counters ctr;                   // the request's counters (stats, hit_count)
    Scratch sc;                     // sc.ctr = &ctr; sc.hits = the slot's hit buffer
    FrameDesc fd;                   // frame constants and caller's output planes
};
static_assert(sizeof(FrameDesc) % 16 == 0, "FrameDesc is copied as uint4");

// One resident request: which control block, published by writing seq last.
struct alignas(16) ServeSlot {
    unsigned long long seq;         // admission sequence (the request's generation); 0 while empty
    unsigned long long prio;        // warps serve the published request with the smallest prio first
    unsigned block;                 // index into the ReqBlock array
    unsigned pad;
};

struct ServeCtl {
    ServeSlot *slots;               // device array of kMaxSlots
    ReqBlock *blocks;               // device array of kReqBlocks
    unsigned *done_flags;           // mapped host memory: generation of the last finished request per slot
    unsigned *exit_flag;            // device memory, 0 at launch: non-zero makes every warp exit
    unsigned *hold;                 // mapped host memory: non-zero while the host has queued or running work
    unsigned long long *times;      // mapped host memory: per slot {first item claimed, finished}, %globaltimer ns
    unsigned long long idle_ns;     // a warp with no work (and no hold) for this long ends the launch
    unsigned long long hold_ns;     // ... and with hold set, after this long regardless
};

cudaError_t serve_launch(const ServeCtl &ctl, int num_sms, cudaStream_t st);

}  // namespace dqj
