// Fused node kernels, double instantiations (see nodes_impl.cuh).
#include "nodes_impl.cuh"

namespace bridge {

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <> cudaError_t launch_node<double>(int n, int batch, const NodeArgs& a, int* grid_used, cudaStream_t s) {
    const int sms = sm_count();
    switch (n) {
        case 16: return node_dispatch<double, 16>(batch, sms, a, s, grid_used);
        case 32: return node_dispatch<double, 32>(batch, sms, a, s, grid_used);
        case 64: return node_dispatch<double, 64>(batch, sms, a, s, grid_used);
        case 128: return node_dispatch<double, 128>(batch, sms, a, s, grid_used);
        case 256: return node_dispatch<double, 256>(batch, sms, a, s, grid_used);
        case 512: return node_dispatch<double, 512>(batch, sms, a, s, grid_used);
        default: return cudaErrorInvalidValue;
    }
}

template <> int node_max_grid<double>(int n, int batch) {
    const int sms = sm_count();
    switch (n) {
        case 16: return node_grid_max<double, 16>(batch, sms);
        case 32: return node_grid_max<double, 32>(batch, sms);
        case 64: return node_grid_max<double, 64>(batch, sms);
        case 128: return node_grid_max<double, 128>(batch, sms);
        case 256: return node_grid_max<double, 256>(batch, sms);
        case 512: return node_grid_max<double, 512>(batch, sms);
        default: return 0;
    }
}

template <> size_t node_scratch_bytes<double>(int n, int batch) {
    const int sms = sm_count();
    switch (n) {
        case 16: return node_scratch_max<double, 16>(batch, sms);
        case 32: return node_scratch_max<double, 32>(batch, sms);
        case 64: return node_scratch_max<double, 64>(batch, sms);
        case 128: return node_scratch_max<double, 128>(batch, sms);
        case 256: return node_scratch_max<double, 256>(batch, sms);
        case 512: return node_scratch_max<double, 512>(batch, sms);
        default: return 0;
    }
}

cudaError_t upload_node_twiddles_f64() { return upload_twiddles_here(); }

}  // namespace bridge
