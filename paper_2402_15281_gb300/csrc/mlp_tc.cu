// mlp_tc.cu -- placeholder until the tcgen05 kernel lands.
#include "mlp_tc.cuh"
namespace svm {
int tc_tile_rows() { return 128; }
size_t tc_workspace_bytes(int) { return 256; }
int tc_prepare(TcModel& t, const svm_model_desc& d, const DevWeights&) { t.prec = d.prec; return 0; }
void tc_release(TcModel& t) { t.ready = false; }
int tc_launch(TcModel&, const CallArgs&, const DevWeights&, int, void*, int, cudaStream_t) { return -1; }
}  // namespace svm
