// Library-wide entry points of the C ABI: status names and version.
#include "common.cuh"

extern "C" const char *upslam_status_string(upslam_status s) {
    switch (s) {
        case UPSLAM_OK: return "ok";
        case UPSLAM_ERR_INVALID_ARG: return "invalid argument";
        case UPSLAM_ERR_CUDA: return "CUDA launch or runtime error";
        case UPSLAM_ERR_DEGENERATE: return "degenerate normal equations";
        case UPSLAM_ERR_NOT_CONVERGED: return "not converged";
        case UPSLAM_ERR_TIMEOUT: return "device-side wait timed out";
        case UPSLAM_ERR_UNSUPPORTED: return "unsupported on this device";
        case UPSLAM_ERR_CAPACITY: return "request exceeds the fixed scratch capacity";
    }
    return "unknown status";
}

extern "C" const char *upslam_version(void) { return "upslam-gb300 0.1 (sm_103a)"; }
