// All-pairs BatMap comparison (the hot loop of Sec. III-B): tile shapes,
// schedule construction and launch.
#pragma once

#include "common.cuh"

namespace bm {

// Tile shapes of the compare kernel.  A CTA of 256 threads owns a tile of
// TR rows x TC columns (each thread 8 rows x MC columns).  Staged shapes
// (stages > 0) stream the column width in stages of KC words through shared
// memory; direct shapes (stages == 0) stream 4-word steps into registers.
struct ShapeDesc {
    uint32_t id;   // 1-based; 0 = automatic
    uint32_t TR, TC, MC, KC, stages;  // (MC: columns per thread)
    double eff;    // relative throughput per padded word-pair (scheduler prior)
};

constexpr int NUM_SHAPES = BATMAP_NUM_SHAPES;
extern const ShapeDesc SHAPES[NUM_SHAPES];

// Number of SMs of the current device (cached).
int device_sms();

// Build the compare work units of one set (fills S->units, longest first,
// and uploads them).  `shape_eff` (NULL = built-in prior) gives the relative
// throughput of each shape (autotuner); `force_shape` (1..NUM_SHAPES) pins
// one shape; target_cost <= 0 picks about 32 units per SM.
void build_schedule(batmap_set *S);
void schedule_units(const batmap_set *S, uint32_t force_shape, const double *shape_eff,
                    double target_cost, std::vector<WorkUnit> *out);

// Width-skewed pairs may be counted by probing (Sec. V's second k-way idea:
// look up the elements of the smaller set in the larger one) instead of the
// cyclic scan.  A probe unit (shape index PROBE_SHAPE) holds consecutive rows
// [r0, r1) of the sorted order and at most PROBE_COLS columns [c0, c1) of one
// width class at least 2^probe_log times wider; one warp visits every
// nonempty slot of each row and reads the one slot of every column that can
// hold the same element (the slot and the code fix pi_t(x)).  It counts
// exactly the slot pairs the scan would count.  Of the rows eligible by
// probe_log, the scheduler probes those where its cost model says probing is
// cheaper than the scan.  probe_log = 0 in batmap_params selects
// PROBE_LOG_DEFAULT; values >= 32 turn the route off.
constexpr uint32_t PROBE_SHAPE = NUM_SHAPES;
constexpr uint32_t PROBE_COLS = 16;
constexpr uint32_t PROBE_LOG_DEFAULT = 2;
uint32_t probe_log_of(const batmap_params &p);  // 0 = route off

// Estimated cost of a unit (padded word-pairs / shape efficiency) and the
// order used by every launch: units of the main shapes first, longest first,
// then those of the one-column shapes 14..16 (small_shape), longest first,
// then the probe units in the order the schedule listed them (column chunk
// by column chunk, so that concurrently probed columns share L2).
double unit_cost(const WorkUnit &u);
void sort_units(std::vector<WorkUnit> *units);
bool small_shape(uint32_t shape);
bool probe_shape(uint32_t shape);
struct UnitParts {
    uint32_t main = 0, small = 0, probe = 0;  // lengths of the three parts, in list order
};
UnitParts unit_parts(const std::vector<WorkUnit> &units);

// Launch the persistent compare kernels over the units at d_units (any mix of
// instances) ordered by sort_units: one kernel per nonempty part, pulling
// work from d_counters[0], [1] and [2] (zeroed by the caller).  Scan kernels
// run one CTA per SM.  d_stamps (optional, set by the caller to {~0, 0})
// receives the earliest CTA start and latest end in globaltimer nanoseconds
// (timing inside captured graphs).  probe_start (optional) is recorded on the
// stream after the scan kernels, before the probe kernel.
void launch_compare(const InstView *d_views, const WorkUnit *d_units, UnitParts parts, uint32_t *d_counters,
                    cudaStream_t st, unsigned long long *d_stamps = nullptr, cudaEvent_t probe_start = nullptr);
constexpr uint32_t COMPARE_COUNTERS = 3;

// Sets the kernel's shared-memory attribute (call before stream capture).
void prepare_compare();

// Shared-memory bytes of one shape (for occupancy and launch).
size_t compare_smem_bytes(uint32_t shape_idx);

}  // namespace bm
