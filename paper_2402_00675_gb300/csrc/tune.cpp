// Per-device table of tuned launch shapes.
#include "tune.h"

#include <map>
#include <mutex>
#include <tuple>

namespace montgb {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, LaunchShape> g_table;  // (device, width, variant, mode)

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return dev;
}
}  // namespace

LaunchShape tuned_shape(int width, int variant, int mode) {
  const auto key = std::make_tuple(current_device(), width, variant, mode);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(key);
  if (it != g_table.end()) return it->second;
  return LaunchShape{};
}

void set_tuned_shape(int width, int variant, int mode, const LaunchShape& shape) {
  const auto key = std::make_tuple(current_device(), width, variant, mode);
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[key] = shape;
}

LaunchShape tuned_batched_shape(int width) {
  // mode -1 marks the batched kernel in the table
  return tuned_shape(width, -1, -1);
}

void set_tuned_batched_shape(int width, const LaunchShape& shape) {
  set_tuned_shape(width, -1, -1, shape);
}

}  // namespace montgb
