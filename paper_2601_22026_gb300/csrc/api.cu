// Host-side helpers of the gsfit C ABI: version, status names, batch layout.
#include "common.cuh"

extern "C" int gsfit_abi_version(void) { return GSFIT_ABI_VERSION; }

extern "C" const char* gsfit_status_string(int code) {
    switch (code) {
        case GSFIT_OK: return "ok";
        case GSFIT_ERR_INVALID_ARG: return "invalid argument";
        case GSFIT_ERR_CAPACITY: return "instance capacity exceeded";
        case GSFIT_ERR_CUDA: return "CUDA error";
        case GSFIT_ERR_TIMEOUT: return "bounded device wait ran out";
        default: return "unknown status";
    }
}

extern "C" int gsfit_camera_layout(gsfit_camera* cams, int n_views, int tile, int32_t* total_tiles,
                                   int64_t* total_pixels) {
    if (!cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || (tile != 8 && tile != 16)) return GSFIT_ERR_INVALID_ARG;
    long long toff = 0, poff = 0;
    for (int v = 0; v < n_views; ++v) {
        if (cams[v].width < 1 || cams[v].height < 1) return GSFIT_ERR_INVALID_ARG;
        const long long tx = (cams[v].width + tile - 1) / tile, ty = (cams[v].height + tile - 1) / tile;
        if (toff > 0x7fffffffll || poff > 0x7fffffffll) return GSFIT_ERR_INVALID_ARG;
        cams[v].tile_offset = (int32_t)toff;
        cams[v].pixel_offset = (int32_t)poff;
        cams[v].tile = tile;
        toff += tx * ty;
        poff += (long long)cams[v].width * cams[v].height;
    }
    if (toff > 0x7fffffffll || poff > 0x7fffffffll) return GSFIT_ERR_INVALID_ARG;
    if (total_tiles) *total_tiles = (int32_t)toff;
    if (total_pixels) *total_pixels = poff;
    return GSFIT_OK;
}
