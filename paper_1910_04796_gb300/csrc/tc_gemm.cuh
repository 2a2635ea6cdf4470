// tc_gemm.cuh -- tensor-core (tcgen05) GEMM kernels of the emulated paths.
#pragma once
#include <cuda.h>

#include "internal.cuh"

namespace dbcsr {

// Work description of one tcgen05 GEMM launch (see tc_ozaki.cu).
struct OzParams {
    int M, N;             // output size
    int kblocks;          // K blocks of 128 bytes (64 bf16 / 32 fp32)
    int s;                // levels d = 2 .. s+1 (slices per operand; 1 for TF32)
    int ksegs;            // K segments (exact int32 accumulation per segment)
    int kseg_blocks;      // k-blocks per segment
    int chunk_blocks;     // k-blocks accumulated in TMEM before the epilogue takes them
    int elem_bytes;       // 2 (bf16 slices) or 4 (tf32)
    int tiles_m, tiles_n;
    int64_t units;        // tiles_m * tiles_n * ksegs * s
    double* ws;           // slices: [s][ksegs][N][M] exact level sums (column-major M x N)
    int64_t ws_stride;    // M * N
    int* ws_i32;          // slices, 256-wide kernel: [s][ksegs][M][ldws] exact int32 level sums (row-major)
    int64_t ldws;         // multiple of 256, >= N
    double* C;            // tf32: output, column-major (ldc), or by rows (cbase, cstride)
    int64_t ldc;
    const int64_t* cbase; // tf32, 256-wide kernel: element (i, j) of C at C[cbase[i] + cstride[i] * j]
    const int* cstride;   //   when cbase is set (C's block storage), else at C[i + j * ldc]
    double alpha, beta;
    int* err;             // set to 1 on a timed-out wait
    uint64_t wait_ns;     // limit of each pipeline wait (ns on the global timer)
};

// FP64 -> FP32 round-to-nearest-even, then FP32 -> TF32 round-to-nearest
// with ties away (cvt.rna.tf32.f32)
__device__ __forceinline__ float to_tf32(double x) {
    const float f = __double2float_rn(x);
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return __uint_as_float(r);
}

int make_slice_tmap(CUtensorMap* map, const void* base, int64_t ldk, int64_t rows, int slices, int box_rows,
                    int elem_bytes);
// slice GEMMs (bf16, 128 x 128 tiles; tmA and tmB boxes of 128 rows) on the library stream
int oz_gemm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p);
// the same on an explicit stream and SM count
int oz_gemm_launch_on(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p, cudaStream_t st,
                      int num_sms);
// TF32 GEMM writing C directly (128 x 128 tiles)
int tf32_gemm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p);

// 128 x 256 tiles (tc_gemm256.cu): usable when its compiled register budget
// matches its warp-group register split; tmB's box then holds 256 rows.
bool tc256_usable();
int oz_gemm256_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p);   // writes ws_i32
int tf32_gemm256_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p);

// 256 x 256 tiles on CTA pairs (tc_gemm2sm.cu): the same int32 level-sum
// workspace as the 128 x 256 kernel; tmA's and tmB's boxes hold 128 rows.
bool tc2sm_usable();
int oz_gemm2sm_launch(const CUtensorMap& tmA, const CUtensorMap& tmB, const OzParams& p);

}  // namespace dbcsr
