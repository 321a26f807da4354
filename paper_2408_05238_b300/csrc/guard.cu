// Guard words around the library's device buffers (a debug mode standing in
// for a memory checker).  While the mode is on, every workspace or factor
// buffer the solver allocates (DevBuf) gets kGuardBytes of a fixed byte
// pattern in front of and behind the bytes it hands out, inside the same
// allocation.  After every kernel launch the library synchronizes the device
// and compares every live buffer's guards with the pattern; a buffer is
// checked once more when it is freed.  A kernel that writes past either end
// of a buffer it was given therefore shows up as a violation naming the
// kernel after which it was seen, without any access leaving the allocation.
// Reads out of bounds are not detected.  The mode serializes the device and
// costs two small copies per buffer per launch: for tests on small shapes.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "lls.h"

namespace lls {

std::atomic<int> g_guard_mode{0};

namespace {

constexpr unsigned char kGuardByte = 0xA5;
constexpr size_t kGuardBytes = 512;  // a multiple of 256: the user pointer keeps cudaMalloc's alignment

struct Region {
  char* base;    // start of the allocation
  size_t bytes;  // bytes handed out, starting at base + kGuardBytes
};

std::mutex g_mu;
std::map<void*, Region> g_regions;  // keyed by the pointer handed out
int64_t g_violations = 0;
std::string g_first;

// Compares both guards of r with the pattern.  Returns "" when intact,
// else a description; a damaged guard is rewritten so that one overrun is
// reported once.
std::string check_region(const Region& r) {
  std::vector<unsigned char> h(kGuardBytes);
  std::string bad;
  for (int side = 0; side < 2; ++side) {
    char* g = side == 0 ? r.base : r.base + kGuardBytes + r.bytes;
    if (cudaMemcpy(h.data(), g, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return "guard read failed";
    }
    size_t first = kGuardBytes, count = 0;
    for (size_t i = 0; i < kGuardBytes; ++i) {
      if (h[i] != kGuardByte) {
        ++count;
        if (first == kGuardBytes) first = i;
      }
    }
    if (count) {
      bad += std::string(side == 0 ? "front" : "back") + " guard of a " + std::to_string(r.bytes) +
             "-byte buffer: " + std::to_string(count) + " bytes changed, first at offset " +
             (side == 0 ? "-" + std::to_string(kGuardBytes - first)
                        : "+" + std::to_string(r.bytes + first)) +
             "; ";
      cudaMemset(g, kGuardByte, kGuardBytes);
      cudaDeviceSynchronize();
    }
  }
  return bad;
}

void record(const std::string& what, const char* after) {
  ++g_violations;
  if (g_first.empty()) g_first = what + "seen after " + (after ? after : "?");
}

}  // namespace

Status guard_alloc(size_t need, void** user) {
  char* base = nullptr;
  if (cudaMalloc(&base, need + 2 * kGuardBytes) != cudaSuccess) {
    cudaGetLastError();
    return make_error(LLS_ERR_NOMEM, "device allocation of " + std::to_string(need) +
                                         " bytes (with guards) failed");
  }
  if (cudaMemset(base, kGuardByte, kGuardBytes) != cudaSuccess ||
      cudaMemset(base + kGuardBytes + need, kGuardByte, kGuardBytes) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(base);
    return make_error(LLS_ERR_CUDA, "guard initialization failed");
  }
  *user = base + kGuardBytes;
  std::lock_guard<std::mutex> lock(g_mu);
  g_regions[*user] = Region{base, need};
  return ok_status();
}

void guard_free(void* user) {
  Region r{};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_regions.find(user);
    if (it == g_regions.end()) return;
    r = it->second;
    std::string bad = check_region(r);
    if (!bad.empty()) record(bad, "the buffer's last use (checked when freed)");
    g_regions.erase(it);
  }
  cudaFree(r.base);
}

void guard_after_launch(const char* name) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& kv : g_regions) {
    std::string bad = check_region(kv.second);
    if (!bad.empty()) record(bad, name);
  }
}

}  // namespace lls

extern "C" int lls_debug_guard(int on) {
  if (on != 0 && on != 1) return LLS_ERR_ARG;
  std::lock_guard<std::mutex> lock(lls::g_mu);
  if (on && !lls::g_guard_mode.load()) {
    lls::g_violations = 0;
    lls::g_first.clear();
  }
  lls::g_guard_mode.store(on);
  return LLS_OK;
}

extern "C" int64_t lls_debug_guard_report(char* msg, int64_t len) {
  std::lock_guard<std::mutex> lock(lls::g_mu);
  if (msg && len > 0) {
    std::strncpy(msg, lls::g_first.c_str(), (size_t)len - 1);
    msg[len - 1] = '\0';
  }
  return lls::g_violations;
}

extern "C" int lls_debug_guard_selftest(void) {
  // A guarded 1000-byte buffer; one byte written just past each end with
  // cudaMemset (inside the allocation) must be reported, an intact buffer
  // must not.  Uses its own region, not the global counters.
  void* user = nullptr;
  lls::Status s = lls::guard_alloc(1000, &user);
  if (!s.ok()) return s.code;
  lls::Region r{};
  {
    std::lock_guard<std::mutex> lock(lls::g_mu);
    r = lls::g_regions[user];
    lls::g_regions.erase(user);
  }
  int code = LLS_OK;
  if (!lls::check_region(r).empty()) code = LLS_ERR_CUDA;
  char* u = static_cast<char*>(user);
  if (code == LLS_OK) {
    cudaMemset(u + 1000, 0, 1);
    cudaDeviceSynchronize();
    std::string bad = lls::check_region(r);
    if (bad.find("back guard") == std::string::npos || bad.find("+1000") == std::string::npos)
      code = LLS_ERR_CUDA;
  }
  if (code == LLS_OK) {
    cudaMemset(u - 3, 0, 2);
    cudaDeviceSynchronize();
    std::string bad = lls::check_region(r);
    if (bad.find("front guard") == std::string::npos || bad.find("-3") == std::string::npos)
      code = LLS_ERR_CUDA;
  }
  if (code == LLS_OK && !lls::check_region(r).empty()) code = LLS_ERR_CUDA;  // rewritten
  cudaFree(r.base);
  return code;
}
