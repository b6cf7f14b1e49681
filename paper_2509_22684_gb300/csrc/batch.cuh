// batch.cuh -- persistent kernel running many transforms (uneven sizes, with
// dependencies between them) in one launch per field.
//
// The paper finds that the Groth16 prover runs seven transforms, every one of
// them as several kernel launches (Section IV-A), and that such short kernels run
// with sub-optimal launch parameters; it calls for runtime autotuning (Section
// V-A).  Here every pass of every transform is a segment of tiles; all tiles of
// all segments form one work list ordered by dependency level.  Resident
// blocks (one grid sized to the SM count) pull the next tile index from a
// device counter.  A segment may depend on up to three earlier segments (the
// previous pass of the same transform, or the producers of its input); the
// block that claims a tile waits until those segments have retired all their
// tiles.  Because tiles are claimed in list order and every dependency points
// to an earlier position, the oldest unfinished tile can always run, so the
// scheme cannot deadlock however many blocks are resident.
//
// Every wait is bounded by `timeout_ns` (device global timer).  On expiry the
// block sets the launch's abort word and the sticky status word, and all blocks
// leave; the host reports ZKNTT_ETIMEOUT.
#pragma once
#include <cstdint>

#include "field.cuh"
#include "ntt_pass.cuh"

namespace zkntt {

constexpr int BATCH_MAX_SEGMENTS = 160;
constexpr uint32_t BATCH_THREADS = 256;
// blocks per SM the register budget is compiled for (64 registers a thread)
#ifndef ZKNTT_BATCH_MIN_BLOCKS
#define ZKNTT_BATCH_MIN_BLOCKS 4
#endif
constexpr int BATCH_MIN_BLOCKS = ZKNTT_BATCH_MIN_BLOCKS;
// resident blocks per SM the tile-width policy counts as one wave
constexpr int BATCH_WAVE_BLOCKS = 3;
// widest batch tile, log2 elements (32 KiB: four blocks per SM fit in shared memory)
constexpr int BATCH_TILE_BITS = 10;
constexpr uint32_t BATCH_STATUS_TIMEOUT = 4u;  // == ZKNTT_ETIMEOUT

struct BatchSeg {
    PassArgs a;
    uint32_t K;           // digit bits of this pass
    uint32_t first_item;  // index of the segment's first tile in the work list
    int32_t dep[3];       // segments that must be complete first (-1: none)
    uint32_t dep_tiles[3];
    uint32_t ntiles;      // tiles in this segment
    uint32_t job;         // index of the transform in the batch
    uint32_t signal;      // 1: last pass of its transform and completion words requested
};

struct BatchTable {
    uint32_t nseg;
    uint32_t total_items;
    unsigned long long timeout_ns;
    uint32_t *flags;      // per-transform completion words (may be null)
    uint32_t epoch;       // value written to flags[job] when the job completes
    BatchSeg seg[BATCH_MAX_SEGMENTS];
};

// passed by value as a kernel parameter (limit 32764 bytes)
static_assert(sizeof(BatchTable) <= 32000, "batch table exceeds the kernel parameter limit");

}  // namespace zkntt
