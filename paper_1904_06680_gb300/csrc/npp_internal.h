// npp_internal.h -- the handle and helpers shared by the host-side
// translation units of the library (not part of the C ABI).
#pragma once

#include <string>

#include <cuda_runtime.h>

#include "../../include/npp.h"
#include "npp_device.cuh"

// collision-kernel variant number of the spatially binned check, and when
// the automatic choice takes it: from 128 points, whatever the number of
// samples (measured on GB300, plan steps at widths 16-64 against the best
// brute-force variant: 1.0-1.3x faster from 128 to 300 points, 1.3-1.8x
// beyond; below 128 points within 2-14 % either way; the grid build runs on
// a side stream while the trajectories are rolled out)
constexpr int COLLIDE_BINNED = 5;
inline bool binned_auto(int M, int N) { (void)N; return M >= 128; }

// the brute-force variant the automatic choice takes otherwise (measured on
// GB300 over M = 20..8000 points and N = 1k..30k samples, every variant
// computing the same flags): with many samples one warp per 8-sample item
// (2) unless the points are many (4: two point slices per item); with few
// samples items on four point slices (3), one warp per item for a handful
// of points, the block-balanced kernel (1) for very many points.  Within 4 %
// of the fastest variant on every measured case.
inline int brute_auto(int M, int N)
{
    if (N >= 6144) return M <= 1200 ? 2 : 4;
    if (M >= 6000) return 1;
    return M <= 64 ? 2 : 3;
}

// most step chunks of one plan step, and the stage events they need
constexpr int NPP_MAX_CHUNKS = 8;
constexpr int NPP_CHUNK_EVENTS = 2 * NPP_MAX_CHUNKS + 1;

struct npp_handle {
    npp_config cfg;
    int device;
    int n_theta;
    int max_points;                      // obstacle points that fit in shared memory
    npp::DevCfg dc;
    unsigned long long* d_key;           // packed best key
    float4* d_traj;                      // [(max_T+1) * max_N]
    float2* d_ctrl;                      // [max_T * max_N]
    float* d_jfree;                      // [max_N]
    int* d_vfirst;                       // [max_N] first speed-violating step (speed limits on)
    float4* d_fp;                        // [FP_MAX_FACES] general footprint faces
    int fp_faces;                        // 0: the rectangle of cfg
    double fp_radius;                    // footprint's largest vertex distance
    unsigned* d_work;                    // persistent-kernel work counter
    int sm_count;
    int collide_variant;                 // -1 automatic, else a fixed collision-kernel variant
                                         // (0..4 brute force, 5 spatially binned)
    int collide_active;                  // variant used for the current launch
    int traj_variant;                    // trajectory launch shape (0..3)
    int fuse;                            // binned check inside the trajectory kernel: -1 automatic
                                         // (at width 64), 0 off, 1 on
    int chunks;                          // step chunks of the binned path when no per-sample records
                                         // are wanted (0: automatic, 1: one launch each)
    int last_chunks;                     // chunks of the last timed plan step (its stage events)
    int* d_live;                         // [2][max_N] samples still collision-free between chunks
    int* d_live_n;                       // [NPP_MAX_CHUNKS] their counts
    float4* d_carry;                     // [max_N] values carried from chunk to chunk
    int loop_restarts;                   // hill-climb rounds per sampling time of new loops (1: none)
    float loop_sigma;                    // their perturbation scale
    int occ_M, occ_blocks;               // cached occupancy for the last M
    float4* d_pXY;                       // EV-frame point pairs when M exceeds shared memory
    unsigned* d_fault;                   // device-wait fault flag of the plan steps (RolloutArgs::fault)
    void* d_bins;                        // per-step spatial grids of the binned collision check
    // host-mode staging
    float4* d_obs;
    float* d_warm;
    float* d_sigma;                      // restart perturbation scale, [n_theta]
    npp_best* d_best;
    float* d_params;
    float* d_controls;
    float* d_trajectory;
    float* d_costs;
    int32_t* d_fh;
    cudaStream_t stream;
    cudaStream_t side;                   // concurrent branch of a plan step (grid build)
    cudaEvent_t fork_ev, join_ev;
    bool timing;
    cudaEvent_t ev[4];                   // start, after trajectories, after collisions, end
    cudaEvent_t cev[NPP_CHUNK_EVENTS];   // chunked step: before trajectories k (2k), before check k
                                         // (2k + 1), after the last check (2K)
    unsigned long long* d_counts;        // measurement counters of the last timed plan step
    std::string err;
};


// cudaEventRecord that becomes a real event-record node under stream capture
// (a plain record there only orders work and is never executed)
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

// p[0 .. n) = v on stream s
cudaError_t fill_floats(float* p, int n, float v, cudaStream_t s);

// records a message for npp_last_error and returns s
npp_status fail(npp_handle* h, npp_status s, const char* fmt, ...);

// stage times of a plan step from its events: [0] trajectories, [1] the
// collision check (each summed over the chunks when nch > 1), [2] the
// epilogue and what follows, [3] the whole step
cudaError_t stage_times(const cudaEvent_t* ev, const cudaEvent_t* cev, int nch, float t[4]);

// trajectory + collision kernels of one plan step (fills workspace pointers,
// the persistent grid and the work-counter reset).  no_records: the caller
// needs no sample's records beyond the winner's, so the binned check may
// run in step chunks or inside the trajectory kernel ("fuse"), which stop
// rolling a sample out after its first collision (the winner's rows, up to
// its first collision, are always complete)
npp_status run_rollout(npp_handle* h, npp::RolloutArgs& a, cudaStream_t s, bool no_records);

#define CUDA_TRY(h, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), NPP_CUDA_ERROR, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
