// ocmc_unet_tc.h -- host entry points of the tcgen05 3x3x3 convolution (ocmc_unet_tc.cu).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ocmc_unet_kernels.cuh"

namespace ocmc {
namespace unet {

// Test hook: from now on every launch's MMA thread, at its block-local tile number `tile`
// (>= 0; -1 turns the hook off), waits `ns` (at most the normal limit) on a barrier that nothing
// completes, so that the wait runs out and the block takes its timeout path.
void conv3_tc_test_stall(int tile, uint64_t ns);

// Channel counts the tensor-memory kernel covers (16 to 128; each block holds the weights of a
// slice of the output channels in shared memory).
bool conv3_tc_supported(int cin, int cout);

// Repack BF16 weights [27][cin][cout] into the kernel's layout [cout/nsl][27][cin/8][nsl][8],
// nsl the kernel's output-channel slice for (cin, cout); for nsl <= 32 the z-taps of each (dx, dy)
// are stacked: [cout/nsl][9][cin/8][3 (dz = 2, 1, 0)][nsl][8].
cudaError_t pack_conv3_tc(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s);

// CONV3 convolution (forward, or data gradient with flipped transposed weights) with the same
// epilogue semantics as k_conv; the input and output grids are a.gin. err (device int, may be
// null) is set to 1 if a wait inside the kernel timed out.
cudaError_t launch_conv3_tc(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s);

// Transposed 2x2x2 convolution (UP, coarse -> fine; also the data gradient of a DOWN layer) on
// the tensor-memory path, for (cin, cout) = (32, 16) and (64, 32). Weights [8][cin][cout]
// are packed by pack_up_tc into [cin/8][8 cout][8]; same epilogue semantics as k_conv's UP mode.
bool up_tc_supported(int cin, int cout);
cudaError_t pack_up_tc(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s);
cudaError_t launch_up_tc(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s);

// Stride-2 2x2x2 convolution (DOWN, fine -> coarse; also the data gradient of an UP layer) on the
// tensor-memory path, for (cin, cout) = (32, 64). Weights [8][cin][cout] are packed
// by pack_down_tc into [8][cin/8][cout][8]; same epilogue semantics as k_conv's DOWN mode.
bool down_tc_supported(int cin, int cout);
cudaError_t pack_down_tc(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s);
cudaError_t launch_down_tc(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s);

// Weight gradient of a 3x3x3 convolution on the tensor-memory path (ocmc_unet_wgrad_tc.cu), for
// (cin, cout) = (16, 16), (32, 16), (16, 32), (32, 32), (64, 32) on grids of at most 128 voxels
// along x whose line stages fit shared memory (wgrad3_tc_fits): dW[t][c][n] = sum over voxels v
// of grid g of x[v + d_t][c] dy[v][n]. Writes one partial [27][cin][cout] per block into part
// (at most part_cap floats) and their count to *parts; the caller sums them in order. err (device
// int, may be null) is set to 1 if a wait inside the kernel timed out.
bool wgrad3_tc_supported(int cin, int cout);
bool wgrad3_tc_fits(int cin, int cout, int nx);
cudaError_t launch_wgrad3_tc(Grid3 g, Slice x, Slice dy, int cin, int cout, float* part, size_t part_cap, int* err,
                             cudaStream_t s, int* parts);

// The CUDA driver's cuTensorMapEncodeTiled (null if the installed driver does not provide it).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

}  // namespace unet
}  // namespace ocmc
