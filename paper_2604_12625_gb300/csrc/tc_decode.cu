#include "tc_decode.h"
namespace ndgi {
bool tc_supported(int, int, int) { return false; }
size_t tc_workspace_bytes(int, int, int) { return 0; }
cudaError_t launch_tc_prepare(const DevModel&, bool, void*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_tc_points(const DevModel&, bool, const void*, const float*, int64_t, float*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_tc_pages(const PagesCtx&, bool, int, int, int, const TcPagesShape&, const ndgi_page_req*, const int32_t*, cudaStream_t) { return cudaErrorNotSupported; }
TcPagesShape tc_default_pages_shape() { return TcPagesShape{1, 16}; }
std::vector<TcPagesShape> tc_pages_candidates(int) { return {TcPagesShape{1, 16}}; }
}
