// Fused node kernels, float instantiations (see nodes_impl.cuh).
#include "nodes_impl.cuh"

namespace bridge {

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <> cudaError_t launch_node<float>(int n, int batch, const NodeArgs& a, int* grid_used, cudaStream_t s) {
    const int sms = sm_count();
    switch (n) {
        case 16: return node_dispatch<float, 16>(batch, sms, a, s, grid_used);
        case 32: return node_dispatch<float, 32>(batch, sms, a, s, grid_used);
        case 64: return node_dispatch<float, 64>(batch, sms, a, s, grid_used);
        case 128: return node_dispatch<float, 128>(batch, sms, a, s, grid_used);
        case 256: return node_dispatch<float, 256>(batch, sms, a, s, grid_used);
        case 512: return node_dispatch<float, 512>(batch, sms, a, s, grid_used);
        default: return cudaErrorInvalidValue;
    }
}

template <> int node_max_grid<float>(int n, int batch) {
    const int sms = sm_count();
    switch (n) {
        case 16: return node_grid_max<float, 16>(batch, sms);
        case 32: return node_grid_max<float, 32>(batch, sms);
        case 64: return node_grid_max<float, 64>(batch, sms);
        case 128: return node_grid_max<float, 128>(batch, sms);
        case 256: return node_grid_max<float, 256>(batch, sms);
        case 512: return node_grid_max<float, 512>(batch, sms);
        default: return 0;
    }
}

template <> size_t node_scratch_bytes<float>(int n, int batch) {
    const int sms = sm_count();
    switch (n) {
        case 16: return node_scratch_max<float, 16>(batch, sms);
        case 32: return node_scratch_max<float, 32>(batch, sms);
        case 64: return node_scratch_max<float, 64>(batch, sms);
        case 128: return node_scratch_max<float, 128>(batch, sms);
        case 256: return node_scratch_max<float, 256>(batch, sms);
        case 512: return node_scratch_max<float, 512>(batch, sms);
        default: return 0;
    }
}

cudaError_t upload_node_twiddles_f32() { return upload_twiddles_here(); }

}  // namespace bridge

namespace bridge {
cudaError_t upload_node_twiddles_f64();
cudaError_t upload_node_twiddles() {
    cudaError_t e = upload_node_twiddles_f32();
    if (e != cudaSuccess) return e;
    return upload_node_twiddles_f64();
}
}  // namespace bridge
