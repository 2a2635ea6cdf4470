// tc_gemm.cuh -- tensor-core (tcgen05) GEMM kernels of the emulated paths.
#pragma once
#include <cuda.h>

#include "internal.cuh"

namespace dbcsr {

// Integer-slice GEMM of the emulated-FP64 product.
struct OzParams {
    int M, N;             // output size
    int kblocks;          // ldk / 64
    int s;                // slices per operand
    int ksegs;            // K segments (exact int32 accumulation per segment)
    int kseg_blocks;      // k-blocks per segment
    int tiles_m, tiles_n;
    int64_t units;        // tiles_m * tiles_n * ksegs * s (levels d = 2 .. s+1)
    double* ws;           // [s][ksegs][N][M] exact level sums (column-major M x N)
    int64_t ws_stride;    // M * N
    int* err;             // set to 1 on a timed-out wait
};

int make_slice_tmap(CUtensorMap* map, const void* base, int64_t ldk, int64_t rows, int slices, int box_rows,
                    int elem_bytes);
int oz_gemm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, int tn);

}  // namespace dbcsr

namespace dbcsr {
// oz_gemm_launch with 128-column tiles on an explicit stream and SM count.
int oz_gemm_launch_on(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, cudaStream_t st,
                      int num_sms);
}  // namespace dbcsr
