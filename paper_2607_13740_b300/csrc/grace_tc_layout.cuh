// Shared-memory image layout of the tensor-core operand tiles.
//
// Operands are stored in global memory already in the canonical K-major,
// 128-byte-swizzled layout that tcgen05.mma reads from shared memory, so a
// whole tile moves with one bulk copy (cp.async.bulk) and needs no tensor map.
//
// A tile covers 128 rows (cells for A, output columns for B) and K elements
// split into "atoms" of 128 bytes per row (32 TF32 or 64 BF16 values).  Atom
// a of a tile with ROWS rows occupies bytes [a*ROWS*128, (a+1)*ROWS*128); in
// it, row r sits at r*128 and its 16-byte chunk c is stored at chunk position
// c ^ (r % 8).  Tiles start on 1024-byte boundaries so the hardware swizzle
// (address bits [4,7) XOR [7,10)) matches this formula.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "grace.h"

namespace grace {

constexpr int kTileM = 128;      // cells per tensor-core tile
constexpr int kAtomBytes = 128;  // swizzle span

__host__ __device__ __forceinline__ int atom_elems(int prec) { return prec == GRACE_TF32 ? 32 : 64; }
__host__ __device__ __forceinline__ int elem_bytes(int prec) { return prec == GRACE_TF32 ? 4 : 2; }
// number of operand planes: TF32 one, BF16X3 two (hi, lo)
__host__ __device__ __forceinline__ int n_planes(int prec) { return prec == GRACE_TF32 ? 1 : 2; }

// byte offset of element (row, k) inside one plane of a tile with `rows` rows
__host__ __device__ __forceinline__ size_t swz_offset(int rows, int row, int k, int ebytes)
{
    const int byte = k * ebytes;
    const int atom = byte >> 7;
    const int inrow = byte & 127;
    const int chunk = (inrow >> 4) ^ (row & 7);
    return (size_t)atom * rows * kAtomBytes + (size_t)row * kAtomBytes + (chunk << 4) + (inrow & 15);
}

// A-operand column of coefficient 0 for P coefficients: the coefficients sit at the end of the
// padded K extent (columns [kofs, kofs + P)), so that the tables' non-zero column ranges, which
// mostly run to the last coefficient, end on a k-step boundary.  Kept a multiple of 16 bytes
// (8 BF16 / 4 TF32 values) so that 16-byte chunks of a row stay aligned.
__host__ __device__ __forceinline__ int a_column_offset(int prec, int P)
{
    const int ae = atom_elems(prec), kpad = (P + ae - 1) / ae * ae, align = 16 / elem_bytes(prec);
    return (kpad - P) / align * align;
}

// bytes of one A tile (128 cells, kpad elements, all planes)
__host__ __device__ __forceinline__ size_t opA_tile_bytes(int prec, int kpad)
{
    return (size_t)kTileM * kpad * elem_bytes(prec) * n_planes(prec);
}

__device__ __forceinline__ uint32_t f32_to_tf32_rna(float f)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

// stores value v (already scaled) of cell `cell`, element k into the A operand
__device__ __forceinline__ void opA_store(void *base, int prec, int kpad, long long cell, int k, double v)
{
    const long long tile = cell / kTileM;
    const int row = (int)(cell - tile * kTileM);
    char *t = (char *)base + (size_t)tile * opA_tile_bytes(prec, kpad);
    if (prec == GRACE_TF32) {
        *(uint32_t *)(t + swz_offset(kTileM, row, k, 4)) = f32_to_tf32_rna((float)v);
    } else {
        const __nv_bfloat16 hi = __double2bfloat16(v);
        const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
        const size_t plane = (size_t)kTileM * kpad * 2;
        *(__nv_bfloat16 *)(t + swz_offset(kTileM, row, k, 2)) = hi;
        *(__nv_bfloat16 *)(t + plane + swz_offset(kTileM, row, k, 2)) = lo;
    }
}

}  // namespace grace
