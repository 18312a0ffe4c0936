// Status strings and build information.
#include "common.cuh"

#define PGSAG_STR2(x) #x
#define PGSAG_STR(x) PGSAG_STR2(x)
#define PGSAG_VIEW_BYTES 152
static_assert(sizeof(pgsag_view) == PGSAG_VIEW_BYTES, "pgsag_view layout");
static_assert(sizeof(pgsag_vote_view) == 96, "pgsag_vote_view layout");
static_assert(sizeof(pgsag_depth_view) == 96, "pgsag_depth_view layout");
static_assert(sizeof(pgsag_tsdf_grid) == 32, "pgsag_tsdf_grid layout");
static_assert(sizeof(pgsag_dssim) == 32, "pgsag_dssim layout");
static_assert(sizeof(pgsag_adam_tensor) == 48, "pgsag_adam_tensor layout");
static_assert(sizeof(pgsag_ban_gather) == 64, "pgsag_ban_gather layout");

extern "C" const char* pgsag_status_str(int status) {
  switch (status) {
    case PGSAG_OK: return "ok";
    case PGSAG_ERR_ARG: return "invalid argument (null pointer, size or alignment)";
    case PGSAG_ERR_CAPACITY: return "capacity or workspace too small";
    case PGSAG_ERR_CUDA: return "CUDA launch or API error";
    case PGSAG_ERR_TIMEOUT: return "bounded device wait expired";
    case PGSAG_ERR_UNSUPPORTED: return "unsupported parameter";
    default: return "unknown status";
  }
}

extern "C" const char* pgsag_build_info(void) {
  return "libpgsag sm_103a; pgsag_view " PGSAG_STR(PGSAG_VIEW_BYTES) " bytes";
}
