// muca_internal.h - launch interface between the host library (muca_api*.cu) and the
// device kernels (muca_kernels.cu and the other kernel files).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace muca {

// Shared-memory table of the whole-sweep kernels: one row of kTableStride words per
// energy, thresholds in words 0..4, the block's histogram count in word kHistSlot.
constexpr int kTableStride = 7;
constexpr int kHistSlot = 5;
// Zero rows below energy 0 and above N for the allocation-free entry point, whose
// energies come from the caller: the threshold candidates loaded ahead of a decision lie
// within two rows of the current energy, so they stay inside the table even for
// energies that do not match the lattices.
constexpr int kTableGuard = 2;
// Table row stride of the batched kernel: 6 words at L = 64 (the histogram word doubles
// as the thermalization padding), so that 256 walkers fit next to the 4097-row table.
__host__ __device__ constexpr int batch_table_stride(int L) { return L == 64 ? 6 : kTableStride; }

// Device error word bits.
constexpr uint32_t kErrEnergyRange = 1u;   // a walker's energy index was off the grid
constexpr uint32_t kErrSyncTimeout = 2u;   // a bounded wait inside a kernel gave up

struct SweepArgs {
    int32_t L;                  // lattice side (multiple of 4, <= 64)
    int32_t layout;             // MUCA_LAYOUT_*
    int64_t W;                  // walkers
    uint64_t seed;              // Philox key
    uint64_t t0;                // attempt counter of the first attempt
    uint64_t n;                 // attempts per walker in this launch
    void *lattice;              // layout-dependent, see muca.h
    int32_t *energy;            // [W]
    const uint32_t *table;      // [(N+1)*5]
    unsigned long long *hist;   // [N+1], accumulated when recording
    uint32_t *err;              // device error word
    const uint32_t *skip = nullptr;   // when set and nonzero at launch: the launch does nothing
    uint32_t walker0 = 0;             // global index of walker 0 (the Philox walker word is walker0 + w)
    // Thermalization attempts run before the launch's n recorded ones, from t0 (the
    // recorded attempts then start at t0 + n_therm).  Only a recording whole-sweep launch
    // (launch_sweep_fused) sets it; every other launch leaves it 0.
    uint64_t n_therm = 0;
};

// Device state of an iteration whose recursion runs on the device (muca_iterate_device).
struct IterState {
    uint32_t done;       // 0: running; 1: the last histogram was flat; 2: iteration limit
    uint32_t update;     // the last metric asked for the recursion and the next table
    int32_t iterations;  // iterations whose histogram was tested
    int32_t prev_lo;     // energy range visited in the previous iteration (-1: none)
    int32_t prev_hi;
    int32_t pad;
    double metric;       // stop metric of the last tested histogram
};

// The steps of one device-side iteration after its recorded sweeps (muca_iterate.cu):
// zeroing the histogram (skipped once done), the stop metric (one block; skipped once
// done), the Eq. (4) recursion and the table of the next iteration (both only when the
// metric kernel set `update`).
cudaError_t launch_iter_reset_hist(unsigned long long *hist, int32_t nb, const IterState *st, cudaStream_t s);
cudaError_t configure_iter_metric(int32_t N);
cudaError_t launch_iter_metric(IterState *st, int32_t N, const unsigned long long *hist, int32_t stop_rule,
                               double flat_threshold, int32_t max_iterations, cudaStream_t s);
cudaError_t launch_iter_recursion(const IterState *st, int32_t N, double *lnW, const unsigned long long *hist,
                                  cudaStream_t s);
cudaError_t launch_iter_table(const IterState *st, int32_t N, const double *lnW, uint32_t *table, cudaStream_t s);

// Thresholds T[e][k] of the weights lnW[N + 1] on the device (the host's build_table
// arithmetic, bit for bit): every weight upload of an instance.
cudaError_t launch_table(int32_t N, const double *lnW, uint32_t *table, cudaStream_t s);

// One work item of the batched kernel: walkers wbase .. wbase + wpb - 1 of instance inst.
struct BatchItem {
    int32_t inst;
    int32_t wpb;
    int64_t wbase;
};

constexpr int kBatchThreads = 256;   // threads per block of the batched kernel

// Shared memory bytes a sweep launch with this many walkers per block needs.
size_t sweep_smem_bytes(int L, int walkers_per_block, bool record);

// Shared memory bytes of the whole-sweep kernel (eight thresholds per energy).
size_t full_smem_bytes(int L, int walkers_per_block, bool record, bool guard = false, int stride = kTableStride);

// Largest dynamic shared memory a block may use on this device (bytes).
size_t sweep_smem_limit();

// Runs attempts [t0, t0 + n) of every walker in one launch: the kernel specialised for
// L (L in {8, 16, 24, 32, 48, 64}; whole sweeps or, with its partial-row path, any
// range), the generic kernel for other L.  Grid = ceil(W / walkers_per_block).
cudaError_t launch_sweep(const SweepArgs &a, int walkers_per_block, bool record, cudaStream_t s);
// a.n_therm thermalization attempts from a.t0, then a.n recorded ones: one launch of the
// whole-sweep kernel where both are whole sweeps from a sweep boundary within one step of
// counter word 1, else a thermalization launch and a recording launch.
cudaError_t launch_sweep_fused(const SweepArgs &a, int walkers_per_block, cudaStream_t s);

// Runs attempts [t0, t0 + n) of every walker in random shared site order (muca_random.cu;
// any L, any attempt range; the given block size, or a smaller one that fits shared
// memory).
cudaError_t launch_random_sweep(const SweepArgs &a, int walkers_per_block, bool record, cudaStream_t s);
size_t random_smem_bytes(int L, int walkers_per_block, bool record);

// Routes whole sweeps to the generic kernel when false (used by tests that compare the
// two kernels).
void set_full_kernel_enabled(bool on);

// Draws the initial spins (tag 1 stream) and their energy indices.
cudaError_t launch_init(int32_t L, int32_t layout, int64_t W, uint64_t seed, uint32_t walker0, void *lattice,
                        int32_t *energy, cudaStream_t s);

// Packs lattices given as int8 in[walker][site] (+1/-1) and recomputes their energies.
cudaError_t launch_pack(int32_t L, int32_t layout, int64_t W, const int8_t *in, void *lattice, int32_t *energy,
                        cudaStream_t s);

// Unpacks lattices into int8 out[walker][site] (+1/-1).
cudaError_t launch_unpack(int32_t L, int32_t layout, int64_t W, const void *lattice, int8_t *out,
                          cudaStream_t s);

// Evaluates the device Philox4x32-10 on n counters.
cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, size_t n, uint32_t *out,
                          cudaStream_t s);

// Kernels of one L each (muca_full_L.cu): launch over any attempt range, and resident
// blocks of the recording kernel per SM.
cudaError_t launch_full_L8(const SweepArgs &a, int wpb, bool record, cudaStream_t s);
cudaError_t launch_full_L16(const SweepArgs &a, int wpb, bool record, cudaStream_t s);
cudaError_t launch_full_L24(const SweepArgs &a, int wpb, bool record, cudaStream_t s);
cudaError_t launch_full_L32(const SweepArgs &a, int wpb, bool record, cudaStream_t s);
cudaError_t launch_full_L48(const SweepArgs &a, int wpb, bool record, cudaStream_t s);
cudaError_t launch_full_L64(const SweepArgs &a, int wpb, bool record, cudaStream_t s);
int occupancy_full_L8(int layout, int wpb);
int occupancy_full_L16(int layout, int wpb);
int occupancy_full_L24(int layout, int wpb);
int occupancy_full_L32(int layout, int wpb);
int occupancy_full_L48(int layout, int wpb);
int occupancy_full_L64(int layout, int wpb);

// Blocks of the recording sweep kernel for this L, layout and block size that one SM
// holds at once (0 if the configuration does not fit).
int resident_blocks(int L, int layout, int walkers_per_block);

// Batched persistent kernel: allows `smem` bytes of dynamic shared memory, reports how
// many blocks of it an SM holds, and launches it over a work list (counter zeroed by
// the caller before every launch; L must be one of 8, 16, 24, 32, 48, 64 and every
// launch covers whole sweeps).
cudaError_t configure_batch(size_t smem);
int batch_resident_blocks(size_t smem);
cudaError_t launch_batch(const SweepArgs *insts, const BatchItem *items, int32_t n_items, uint32_t *counter,
                         int grid, size_t smem, bool record, cudaStream_t s);
// The recording instantiation of the batched kernel (its own translation unit).
cudaError_t configure_batch_record(size_t smem);
int batch_resident_blocks_record(size_t smem);
cudaError_t launch_batch_record(const SweepArgs *insts, const BatchItem *items, int32_t n_items, uint32_t *counter,
                                int grid, size_t smem, cudaStream_t s);

// Allocation-free batched sweep (see muca_batch_sweep_noalloc in muca.h): descriptors,
// walkers per item and the prefix sums of the work items per instance (prefix[0] = 0,
// prefix[n] = all items, below 2^31) come from the host and travel in the launch
// parameters; the kernel's only scratch, its work counter, is a file-scope device array
// of kNoAllocScratchBytes, looked up on the first call per device.
constexpr int kNoAllocMaxInstances = 64;
constexpr int kNoAllocMaxDevices = 64;
constexpr size_t kNoAllocScratchBytes = 256;
cudaError_t launch_batch_noalloc(const SweepArgs *descs, const int32_t *wpbs, const int32_t *prefix, int32_t n,
                                 size_t smem, bool record, cudaStream_t s);

// Issue rate of one instruction class (muca_probe.cu, see muca_measure_issue_rate).
cudaError_t measure_issue_rate(int kind, double *per_second);

// Bytes of the lattice storage of W walkers.
size_t lattice_bytes(int32_t L, int32_t layout, int64_t W);

}  // namespace muca
