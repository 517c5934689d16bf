// Autotuning cache: kernel configurations measured on the device, keyed by the shape of the
// work, kept per context and optionally in a JSON file so that a later process starts from
// them.  The tuned kernel is the Chebyshev step (cheb.cu, the solve's dominant kernel): its
// shared-memory stage budget (which trades L1 room for the gathers in flight against staged
// indices) and whether it loads each row's own blocks before its gathers.  Every
// configuration computes the same values in the same order, so tuning changes times only.
//
// File format: one JSON object, key -> {"budget": bytes, "prefetch": 0|1, "us": time}.
#include "mge_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

namespace mge {

bool tune_lookup(Ctx* ctx, const std::string& key, TuneEntry* e) {
  std::lock_guard<std::mutex> lock(ctx->tune_mu);
  auto it = ctx->tune.find(key);
  if (it == ctx->tune.end()) return false;
  *e = it->second;
  return true;
}

static void tune_save_locked(Ctx* ctx) {
  if (ctx->tune_path.empty()) return;
  const std::string tmp = ctx->tune_path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : ctx->tune) {
    fprintf(f, "  \"%s\": {\"budget\": %d, \"prefetch\": %d, \"us\": %.3f}%s\n", kv.first.c_str(),
            kv.second.budget, kv.second.prefetch, kv.second.us, ++i < ctx->tune.size() ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
  std::rename(tmp.c_str(), ctx->tune_path.c_str());
}

void tune_store(Ctx* ctx, const std::string& key, const TuneEntry& e) {
  std::lock_guard<std::mutex> lock(ctx->tune_mu);
  ctx->tune[key] = e;
  tune_save_locked(ctx);
}

// Reads the entries of a file written by tune_save_locked (keys without quotes or escapes).
static mge_status tune_parse(const std::string& text, std::map<std::string, TuneEntry>* out) {
  size_t p = 0;
  for (;;) {
    const size_t q0 = text.find('"', p);
    if (q0 == std::string::npos) break;
    const size_t q1 = text.find('"', q0 + 1);
    if (q1 == std::string::npos) return MGE_EINVAL;
    const std::string key = text.substr(q0 + 1, q1 - q0 - 1);
    const size_t b0 = text.find('{', q1), b1 = text.find('}', q1);
    if (b0 == std::string::npos || b1 == std::string::npos || b1 < b0) return MGE_EINVAL;
    const std::string body = text.substr(b0, b1 - b0 + 1);
    TuneEntry e;
    const char* s = body.c_str();
    const char* pb = strstr(s, "\"budget\":");
    const char* pp = strstr(s, "\"prefetch\":");
    const char* pu = strstr(s, "\"us\":");
    if (!pb || !pp || !pu) return MGE_EINVAL;
    e.budget = (int)strtol(pb + 9, nullptr, 10);
    e.prefetch = (int)strtol(pp + 11, nullptr, 10);
    e.us = strtod(pu + 5, nullptr);
    if (e.budget <= 0 || (e.prefetch != 0 && e.prefetch != 1)) return MGE_EINVAL;
    (*out)[key] = e;
    p = b1 + 1;
  }
  return MGE_OK;
}

mge_status tune_set(Ctx* ctx, int mode, const char* path) {
  if (mode < 0 || mode > 2) return MGE_EINVAL;
  std::map<std::string, TuneEntry> loaded;
  if (path && *path) {
    FILE* f = fopen(path, "r");
    if (f) {
      std::string text;
      char buf[4096];
      size_t k;
      while ((k = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
      fclose(f);
      const mge_status s = tune_parse(text, &loaded);
      if (s != MGE_OK) {
        set_error(ctx, "autotune cache %s is not in the expected format", path);
        return s;
      }
    }
  }
  std::lock_guard<std::mutex> lock(ctx->tune_mu);
  ctx->tune_mode = mode;
  ctx->tune_path = path ? path : "";
  for (const auto& kv : loaded) ctx->tune[kv.first] = kv.second;
  return MGE_OK;
}

}  // namespace mge
