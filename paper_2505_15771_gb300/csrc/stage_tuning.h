// Launch parameters of the ERK stage kernels, per arithmetic and polynomial
// degree k (array index k - 1):
//   min_blocks  resident 128-thread blocks per SM asked of the register
//               allocator (__launch_bounds__): 8 allow 64 registers a
//               thread, 6 allow 80, 5 allow 96, 4 allow 128;
//   acc_smem    1: the cell's rate accumulators live in dynamic shared
//               memory instead of registers;
//   prefetch    mask of L2 prefetch hints (bits in stage.cu, L2Prefetch);
//   rect_loop   1: a rectangle's faces are traced by one body per
//               orientation looped over its two faces (compact code, fewer
//               live registers); 0: four unrolled bodies with constant signs.
// tune.py (beside the package) rewrites these tables from timings of
// candidate builds on the target GPU; the values here are the fastest it
// and the earlier sweeps found on GB300 for the 1024 x 512 bilayer (FP64,
// double-float) and the batched hybrid and basin meshes (FP32).
#pragma once

struct StageTuning {
    int min_blocks[3];
    int acc_smem[3];
    int prefetch[3];
    int rect_loop[3];
};

// tune.py: begin tables
constexpr StageTuning TUNED_F64 = {{8, 8, 8}, {0, 1, 0}, {0, 50, 0}, {0, 0, 0}};
constexpr StageTuning TUNED_F32 = {{8, 10, 8}, {0, 1, 1}, {50, 50, 50}, {0, 0, 0}};
constexpr StageTuning TUNED_F2X = {{8, 5, 5}, {0, 1, 0}, {0, 50, 0}, {1, 1, 1}};
// tune.py: end tables
