// Stable least-significant-digit radix sort of (64-bit key, 32-bit value)
// pairs on the device, used by the linear BVH builds (lbvh.cu) to order
// items along their Morton curve.  Off the hot path: it runs in
// qrt_scene_create.
//
// Eight bits per pass.  A first kernel reduces the keys to the OR and the
// AND of all of them, and a pass runs only for a digit that is not the same
// in every key (Morton codes of a flat or clustered scene leave whole digits
// constant).  Each pass: per-tile digit counts (tiles of kSortTile
// consecutive items), one exclusive scan over the counts laid out digit-major
// (digit d of tile t at d * tiles + t, so the scan gives every tile's
// first output position for each digit in stable order), and a scatter in
// which every tile ranks its items by (digit, position) in shared memory and
// writes them out in runs of equal digits.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace qrt {

// Bytes of device scratch sort_pairs needs for n pairs.
size_t sort_pairs_scratch_bytes(uint32_t n);

// Sorts the n pairs (keys[i], vals[i]) by bits [0, end_bit) of the key,
// stably (pairs with equal sorting bits keep their input order), and leaves
// the result in keys_out / vals_out.  keys / vals are overwritten (they are
// the second buffer of the ping-pong).  scratch: sort_pairs_scratch_bytes(n)
// bytes of device memory, 16-byte aligned.  The stream is synchronised once,
// after the OR/AND reduction, to read which digits vary.  end_bit in
// [0, 64]; end_bit 0 or n <= 1 copies the input; n at most 2^32 - 2049.
// Returns cudaErrorInvalidValue for an end_bit or n out of range, else the
// first CUDA error.
cudaError_t sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_out, uint32_t* vals_out,
                       uint32_t n, int end_bit, void* scratch, cudaStream_t stream);

}  // namespace qrt
