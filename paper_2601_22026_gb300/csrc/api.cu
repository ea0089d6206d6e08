// Host-side helpers of the gsfit C ABI: version, status names, batch layout,
// view selection for continual refinement.
#include <cmath>

#include "common.cuh"

extern "C" int gsfit_abi_version(void) { return GSFIT_ABI_VERSION; }

extern "C" const char* gsfit_status_string(int code) {
    switch (code) {
        case GSFIT_OK: return "ok";
        case GSFIT_ERR_INVALID_ARG: return "invalid argument";
        case GSFIT_ERR_CAPACITY: return "instance capacity exceeded";
        case GSFIT_ERR_CUDA: return "CUDA error";
        case GSFIT_ERR_TIMEOUT: return "bounded device wait ran out";
        case GSFIT_ERR_NONFINITE: return "non-finite gradient";
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

// Eq. 1 of Section 4.2: novel iff every view of the set is farther than
// delta_pos in position or more than theta_view away in direction.
extern "C" int gsfit_view_is_novel(const float* pos_new, const float* dir_new, const float* pos_set,
                                   const float* dir_set, int32_t n_set, float delta_pos, float cos_theta) {
    if (!pos_new || !dir_new || n_set < 0 || (n_set > 0 && (!pos_set || !dir_set))) return GSFIT_ERR_INVALID_ARG;
    const double ln = std::sqrt((double)dir_new[0] * dir_new[0] + (double)dir_new[1] * dir_new[1] +
                                (double)dir_new[2] * dir_new[2]);
    if (!(ln > 0.0)) return GSFIT_ERR_INVALID_ARG;
    for (int i = 0; i < n_set; ++i) {
        const float* p = pos_set + 3 * i;
        const float* d = dir_set + 3 * i;
        const double li = std::sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
        if (!(li > 0.0)) return GSFIT_ERR_INVALID_ARG;
        const double dx = (double)pos_new[0] - p[0], dy = (double)pos_new[1] - p[1], dz = (double)pos_new[2] - p[2];
        const bool far = std::sqrt(dx * dx + dy * dy + dz * dz) > (double)delta_pos;
        const double cosang = ((double)dir_new[0] * d[0] + (double)dir_new[1] * d[1] + (double)dir_new[2] * d[2]) /
                              (ln * li);
        const bool turned = cosang < (double)cos_theta;
        if (!(far || turned)) return 0;  // close to view i in both position and direction
    }
    return 1;
}
