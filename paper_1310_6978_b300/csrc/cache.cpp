// cache.cpp -- process-wide caches of the host compiler's products.
//
// Compiling the same text again (a service that sees a recurring query, a
// loop that recompiles its formula) repeats work whose result depends only
// on the text, the domain size and the kernel-shape options: parsing and
// grounding (the map * of Sec. 3.1 and the Reduction of Sec. 4.1), the
// layout, the lowering to LUTs, the build-time item pruning and the emitted
// source or bytecode.  These caches keep the most recent results, immutable
// and shared; device buffers stay per program.
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "build_cache.hpp"
#include "program.hpp"

namespace fbg {

namespace {

// A bounded map from key to shared immutable value; the oldest insertion is
// dropped first.
template <class V>
class SharedCache {
 public:
  explicit SharedCache(size_t cap) : cap_(cap) {}
  std::shared_ptr<const V> get(const std::string& key) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = map_.find(key);
    if (it == map_.end()) {
      misses_++;
      return nullptr;
    }
    hits_++;
    return it->second;
  }
  void put(const std::string& key, std::shared_ptr<const V> v) {
    // entries dropped here are destroyed after the lock is released, so that
    // freeing a large build does not hold up other threads' lookups
    std::vector<std::shared_ptr<const V>> dropped;
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (map_.count(key)) return;
      map_.emplace(key, std::move(v));
      order_.push_back(key);
      while (order_.size() > cap_) {
        auto it = map_.find(order_.front());
        if (it != map_.end()) {
          dropped.push_back(std::move(it->second));
          map_.erase(it);
        }
        order_.pop_front();
      }
    }
  }
  void clear() {
    std::lock_guard<std::mutex> lk(mu_);
    map_.clear();
    order_.clear();
  }
  void stats(uint64_t* hits, uint64_t* misses, uint64_t* entries) {
    std::lock_guard<std::mutex> lk(mu_);
    *hits = hits_;
    *misses = misses_;
    *entries = map_.size();
  }

 private:
  size_t cap_;
  std::mutex mu_;
  std::unordered_map<std::string, std::shared_ptr<const V>> map_;
  std::deque<std::string> order_;
  uint64_t hits_ = 0, misses_ = 0;
};

SharedCache<Compiled>& compiled_cache() {
  static SharedCache<Compiled> c(512);
  return c;
}
SharedCache<JitHost>& jit_cache() {
  static SharedCache<JitHost> c(256);
  return c;
}
SharedCache<JitDevice>& jit_device_cache() {
  static SharedCache<JitDevice> c(512);
  return c;
}
SharedCache<InterpHost>& interp_cache() {
  static SharedCache<InterpHost> c(512);
  return c;
}

}  // namespace

std::shared_ptr<const Compiled> compile_cached(const std::string& text, int k) {
  const std::string key = std::to_string(k) + "\n" + text;
  if (auto hit = compiled_cache().get(key)) return hit;
  auto c = std::make_shared<Compiled>();
  c->th = parse_theory(text, k);
  c->g = ground(c->th);
  std::shared_ptr<const Compiled> cc = std::move(c);
  compiled_cache().put(key, cc);
  return cc;
}

std::string build_key(const fbg_program* p, const char* what, int mode) {
  std::string key = what;
  key += ":" + std::to_string(mode);
  for (int64_t v : {p->opt_prune, p->opt_regs_log2, p->opt_warps_log2, p->opt_unit_bits, p->opt_loop_level_bits,
                    p->opt_search, p->opt_min_blocks, p->opt_stats, p->opt_inner_bits, p->opt_popc_cost,
                    p->opt_order_seed})
    key += ":" + std::to_string(v);
  key += ":" + std::to_string(p->k) + "\n" + p->text;
  return key;
}

std::shared_ptr<const JitHost> jit_host_get(const std::string& key) { return jit_cache().get(key); }
void jit_host_put(const std::string& key, std::shared_ptr<const JitHost> v) { jit_cache().put(key, std::move(v)); }
std::shared_ptr<const InterpHost> interp_host_get(const std::string& key) { return interp_cache().get(key); }
void interp_host_put(const std::string& key, std::shared_ptr<const InterpHost> v) {
  interp_cache().put(key, std::move(v));
}

std::shared_ptr<JitDevice> jit_device_get(const std::string& key, int device) {
  auto v = jit_device_cache().get(std::to_string(device) + "#" + key);
  return std::const_pointer_cast<JitDevice>(v);
}
void jit_device_put(const std::string& key, int device, std::shared_ptr<JitDevice> v) {
  jit_device_cache().put(std::to_string(device) + "#" + key, std::move(v));
}

void host_caches_clear() {
  compiled_cache().clear();
  jit_cache().clear();
  jit_device_cache().clear();
  interp_cache().clear();
}

void host_cache_stats(uint64_t out[9]) {
  compiled_cache().stats(&out[0], &out[1], &out[2]);
  jit_cache().stats(&out[3], &out[4], &out[5]);
  interp_cache().stats(&out[6], &out[7], &out[8]);
}

}  // namespace fbg
