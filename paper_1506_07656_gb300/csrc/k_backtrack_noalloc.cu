// Backtracking and reciprocal verification for callers that cannot allocate
// device memory (dm_backtrack_noalloc in include/dm.h).
//
// Some callers cannot give the library a workspace: plug-ins that run inside a
// host application which owns all device memory and forbids allocations after
// start-up, or loops that must never call cudaMalloc because it can
// synchronise the device.  For them the scratch of the backtracking step (the
// per-level merge tables, the BestAt / BestAt' keys and the
// status header) lives in one fixed, file-scope device array instead of a
// caller workspace.  The kernels are the ones dm_backtrack launches; only the
// memory they are given differs.
//
// The array costs DM_NOALLOC_SCRATCH_BYTES on every GPU that loads the
// library, for as long as the process lives.  In host code its name is only a
// host-side stand-in: its device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <mutex>
#include <string>

#include "dm_internal.cuh"

static __device__ __align__(256) unsigned char g_bt_scratch[DM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices];   // device address of g_bt_scratch per device (null = not set up)

// Device address of the scratch array on `device` (which must be current).
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (g_scratch_ptr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bt_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

// Makes `d` the current device for the scope of one call and restores the
// previous one; ok() is false when `d` could not be made current.
struct DeviceScope {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int d) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != d) {
            err = cudaSetDevice(d);
            changed = err == cudaSuccess;
        }
    }
    bool ok() const { return err == cudaSuccess; }
    ~DeviceScope() {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" dm_status dm_backtrack_noalloc(dm_ctx* ctx, const dm_pyramid* pyr, dm_match_t* d_out, int capacity,
                                          int* d_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!pyr || !d_out || !d_count || capacity < 0)
        return dm_set_error(ctx, DM_EINVAL, "dm_backtrack_noalloc: bad arguments");
    DmBtLayout bl;
    dm_bt_layout(pyr->g, &bl);
    if (bl.bytes > (size_t)DM_NOALLOC_SCRATCH_BYTES) {
        std::string msg = "dm_backtrack_noalloc: this pair needs " + std::to_string(bl.bytes) +
                          " bytes of backtracking scratch, more than the fixed " +
                          std::to_string((size_t)DM_NOALLOC_SCRATCH_BYTES) + " bytes; use dm_backtrack";
        return dm_set_error(ctx, DM_ENOMEM, msg.c_str());
    }
    DeviceScope scope(dm_ctx_device(ctx));
    if (!scope.ok()) {
        // the array's address must be taken with the context's device current
        std::string msg = std::string("dm_backtrack_noalloc: cannot make the context's device current: ") +
                          cudaGetErrorString(scope.err);
        return dm_set_error(ctx, DM_ECUDA, msg.c_str());
    }
    void* scratch = nullptr;
    cudaError_t e = scratch_address(dm_ctx_device(ctx), &scratch);
    if (e != cudaSuccess) {
        std::string msg = std::string("dm_backtrack_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return dm_set_error(ctx, DM_ECUDA, msg.c_str());
    }
    // dm_launch_backtrack clears the header and the BestAt / BestAt' keys, and
    // each level's active table, before use, so nothing of an earlier call leaks.
    e = dm_launch_backtrack(pyr->g, *pyr, bl, static_cast<char*>(scratch), d_out, capacity, d_count,
                            (cudaStream_t)stream);
    if (e != cudaSuccess) {
        std::string msg = std::string("dm_backtrack_noalloc: ") + cudaGetErrorString(e);
        return dm_set_error(ctx, DM_ECUDA, msg.c_str());
    }
    return DM_OK;
}
