// Shared pieces of the tcgen05 Gram kernels (gram_tc.cu, gram_fused.cu): tile constants, the
// shared-memory control block and the quad-unit work schedule (internal header).
#pragma once

#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dfs {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_ROW_BYTES = 128;
constexpr int TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_BM * TC_ROW_BYTES;  // one 128-row tile of one k-block
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;    // A0, A1, B0, B1
constexpr int TC_PART = 2 * TC_BM * TC_BN;            // floats per partial block
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcSmem {
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t accf;
    uint64_t acce;
    uint64_t done;
    uint32_t tmem_base;
    int abort;
    int never;  // stays 0: the abort flag for waits that must not be cut short
};

constexpr size_t TC_SMEM_BYTES = 1024 + (size_t)TC_STAGES * TC_STAGE_BYTES + sizeof(TcSmem);

// Warp roles: warp 0 producer, warp 1 MMA issuer, warps 2-5 epilogue.
constexpr int TC_THREADS = 192;
constexpr int kMmaWarp = 1;

// Units (I2, J2), J2 <= I2 < T2, in row-major order: unit u = I2 (I2 + 1) / 2 + J2.
__host__ __device__ __forceinline__ void tc_unit_ij(int u, int& I2, int& J2) {
    int i = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= u) ++i;
    while (i * (i + 1) / 2 > u) --i;
    I2 = i;
    J2 = u - i * (i + 1) / 2;
}

// The unit list: all (I2, J2), J2 <= I2 < T2, in row-major order when H2 = 0; for the stacked
// BF16x3 operand (H2 > 0, T = 4 H2) the H H^T triangle (I2 < H2, row-major) followed by the L H^T
// rectangle (I2 >= H2, J2 < H2, row-major).
__host__ __device__ __forceinline__ int tc_num_units(int T, int H2) {
    const int T2 = (T + 1) / 2;
    return H2 ? H2 * (H2 + 1) / 2 + H2 * H2 : T2 * (T2 + 1) / 2;
}
__host__ __device__ __forceinline__ void tc_unit_ij2(int u, int H2, int& I2, int& J2) {
    const int tri = H2 * (H2 + 1) / 2;
    if (H2 == 0 || u < tri) {
        tc_unit_ij(u, I2, J2);
        return;
    }
    I2 = H2 + (u - tri) / H2;
    J2 = (u - tri) % H2;
}
__host__ __device__ __forceinline__ int tc_unit_index(int I2, int J2, int H2) {
    if (H2 == 0 || I2 < H2) return I2 * (I2 + 1) / 2 + J2;
    return H2 * (H2 + 1) / 2 + (I2 - H2) * H2 + J2;
}

struct TcTask {
    int I2, J2, slot, stride;
};
// Group gi -> unit gi mod U and slot group gi / U; its t-th task takes slot (gi / U) G + t, i.e.
// the k-blocks slot, slot + c, slot + 2c, ...
__host__ __device__ __forceinline__ TcTask tc_task(int gi, int t, int U, int c, int G, int H2) {
    TcTask k;
    tc_unit_ij2(gi % U, H2, k.I2, k.J2);
    k.slot = (gi / U) * G + t;
    k.stride = c;
    return k;
}

__host__ __device__ __forceinline__ int tc_task_nk(const TcTask& k, int64_t nkb) {
    return k.slot < nkb ? (int)((nkb - 1 - k.slot) / k.stride + 1) : 0;
}

}  // namespace dfs
