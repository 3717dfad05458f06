// mgs_quantize_groups_noalloc: the codes of one chosen configuration without
// any device allocation.  The only scratch it needs (the kept list of the
// chosen kept-set size and the per-tile counts that build it) lives in the
// file-scope device arrays below, which every GPU that loads this library
// holds for the life of the process.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

// MGS_NOALLOC_MAX_KEEP kept indices (16 MiB) and the tile counts of a scene of up
// to MGS_NOALLOC_MAX_SCENE Gaussians (16 KiB).
static __device__ __align__(256) int32_t g_noalloc_kept[MGS_NOALLOC_MAX_KEEP];
constexpr int64_t kNoallocTiles = mgs::kept_tiles_for(MGS_NOALLOC_MAX_SCENE);
static __device__ __align__(256) uint32_t g_noalloc_tiles[kNoallocTiles];
static_assert(kNoallocTiles * mgs::kKeptTile >= MGS_NOALLOC_MAX_SCENE,
              "one tile count per kept-list tile of the largest scene");

constexpr int kMaxDevices = 64;

struct DeviceScratch {
    std::once_flag once;
    cudaError_t status = cudaSuccess;
    int32_t *kept = nullptr;
    uint32_t *tiles = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];

// Device addresses of the arrays on the current device (looked up once per device;
// in host code the arrays' names are only host-side handles).
mgs_status scratch_for(int device, int32_t **kept, uint32_t **tiles) {
    if (device < 0 || device >= kMaxDevices) {
        mgs::set_error("device %d outside 0..%d", device, kMaxDevices - 1);
        return MGS_ERR_INVALID_ARG;
    }
    DeviceScratch &d = g_scratch[device];
    std::call_once(d.once, [&] {
        d.status = cudaGetSymbolAddress((void **)&d.kept, g_noalloc_kept);
        if (d.status == cudaSuccess) d.status = cudaGetSymbolAddress((void **)&d.tiles, g_noalloc_tiles);
    });
    if (d.status != cudaSuccess) {
        mgs::set_error("cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(d.status));
        return MGS_ERR_CUDA;
    }
    *kept = d.kept;
    *tiles = d.tiles;
    return MGS_OK;
}

}  // namespace

extern "C" mgs_status mgs_quantize_groups_noalloc(mgs_ctx *ctx, const mgs_scene *scene,
                                                  int64_t keep, int32_t group_size,
                                                  const uint8_t *bits, uint16_t *codes,
                                                  float *minmax, void *stream) {
    mgs::clear_error();
    if (!ctx || !scene || !bits || !codes || !minmax) {
        mgs::set_error("ctx, scene, bits, codes and minmax must be non-NULL");
        return MGS_ERR_INVALID_ARG;
    }
    if (keep < 1 || keep > scene->n || group_size < 1 || group_size > MGS_MAX_GROUP) {
        mgs::set_error("keep %lld or group_size %d out of range", (long long)keep, group_size);
        return MGS_ERR_INVALID_ARG;
    }
    if (keep > MGS_NOALLOC_MAX_KEEP || scene->n > MGS_NOALLOC_MAX_SCENE) {
        mgs::set_error("mgs_quantize_groups_noalloc holds at most %d kept Gaussians of a scene of "
                       "at most %d (asked: keep %lld of %lld); use mgs_quantize_groups",
                       MGS_NOALLOC_MAX_KEEP, MGS_NOALLOC_MAX_SCENE, (long long)keep,
                       (long long)scene->n);
        return MGS_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) {
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) {
            mgs::set_error("cudaSetDevice(%d): %s", ctx->device, cudaGetErrorString(e));
            return MGS_ERR_CUDA;
        }
    }
    int32_t *kept = nullptr;
    uint32_t *tiles = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mgs_status s = scratch_for(ctx->device, &kept, &tiles);
    if (s == MGS_OK) s = mgs::kept_list_into(scene, keep, kept, tiles, st);
    if (s == MGS_OK)
        s = mgs::quantize_launch(ctx, scene, kept, keep, group_size, bits, codes, minmax, st);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return s;
}
