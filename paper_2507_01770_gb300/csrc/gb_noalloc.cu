// gb_eval_boxes_noalloc: the per-box evaluation of gb_eval_boxes for callers
// that cannot allocate device memory while they run -- for example a serving
// process that has already handed all free device memory to its own pool, or
// a latency-critical thread that must not wait on the device allocator.
//
// gb_eval_boxes asks the stream-ordered allocator for a scratch buffer that
// holds the boxes rounded outward to float (FP32 mode).  This entry point
// keeps that scratch in the fixed array below instead.  The array is part of
// the library's device image, so every GPU that loads the library holds it
// (8 MiB) until the process exits.  Host code cannot use the array's name as
// a device address: the address is looked up per device with
// cudaGetSymbolAddress, with that device current, on the first FP32 call
// (retried on later calls until a lookup succeeds).  The FP64 mode needs no
// scratch and never touches the array.
#include <cuda_runtime.h>

#include <mutex>

#include "gb_internal.h"
#include "gb_launch.h"

#define GB_NOALLOC_MAX_COORDS (1 << 20)   // nbox * n coordinates per FP32 call
#define GB_NOALLOC_MAX_DEVICES 64

namespace {

// A call with nbox boxes of n coordinates uses [0, nbox * n) for the lower
// bounds as floats and [nbox * n, 2 * nbox * n) for the upper bounds.  Every
// call writes the part it reads before reading it, so nothing needs clearing.
static __device__ __align__(256) float g_noalloc_scratch[2 * GB_NOALLOC_MAX_COORDS];

std::mutex g_mu;
float* g_ptr[GB_NOALLOC_MAX_DEVICES];   // set only by a successful lookup

// This device's copy of the array (the device must be current); null if the
// lookup fails (the next call tries again).
float* scratch_of(int device) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[device]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) == cudaSuccess) g_ptr[device] = (float*)ptr;
        else cudaGetLastError();   // do not leave the failed lookup as the thread's pending error
    }
    return g_ptr[device];
}

}  // namespace

extern "C" gb_status gb_eval_boxes_noalloc(gb_problem* prob, const double* d_lo, const double* d_hi,
                                           int64_t nbox, int32_t blk, int32_t fp32, double* d_F,
                                           double* d_Fmid, double* d_G, int32_t* d_mono, void* stream) {
    int device = 0, n = 0, nb = 0;
    const GbProg* P = gb_internal_prog(prob, &device, &n, &nb);
    if (!P) return gb_internal_fail(GB_E_INVALID, "NULL problem");
    if (nbox < 0 || blk >= nb || (nbox > 0 && (!d_lo || !d_hi || !d_F || !d_Fmid)) ||
        (blk >= 0 && nbox > 0 && (!d_G || !d_mono)))
        return gb_internal_fail(GB_E_INVALID, "bad arguments to gb_eval_boxes_noalloc");
    if (fp32 && nbox > 0 && nbox > (int64_t)GB_NOALLOC_MAX_COORDS / n)
        return gb_internal_fail(GB_E_INVALID,
                                "gb_eval_boxes_noalloc: nbox * n exceeds the fixed FP32 scratch of 2^20 coordinates");
    if (device < 0 || device >= GB_NOALLOC_MAX_DEVICES)
        return gb_internal_fail(GB_E_INVALID, "gb_eval_boxes_noalloc: device ordinal above 63");
    if (nbox == 0) return GB_OK;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return gb_internal_fail(GB_E_CUDA, "cudaSetDevice failed");
    gb_status rc = GB_OK;
    float* scratch = nullptr;
    if (fp32 && !(scratch = scratch_of(device))) {
        rc = gb_internal_fail(GB_E_CUDA, "gb_eval_boxes_noalloc: cudaGetSymbolAddress failed");
    } else {
        cudaError_t e = gb_launch_eval_boxes(*P, d_lo, d_hi, scratch, nbox, blk, fp32, d_F, d_Fmid, d_G, d_mono,
                                             (cudaStream_t)stream);
        if (e != cudaSuccess) rc = gb_internal_fail(GB_E_CUDA, cudaGetErrorString(e));
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);   // leave the caller's current device as it was
    return rc;
}
