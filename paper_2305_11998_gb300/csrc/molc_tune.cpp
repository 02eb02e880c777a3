// Tuning cache of MOLC_AUTOTUNE (see molc_tune.h): a small JSON reader and writer for the cache file, and the
// process-wide cache behind molc_tune_cache.
//
// File format (written by tune_serialize, read back by tune_parse):
//   {"format": "molc-tune-cache", "version": 1,
//    "entries": [{"key": "...", "device": "...", "build": "...", "sweep_depth": 4, "tile_cells": 0,
//                 "tile_groups": 0, "block_threads": 0, "best_ms": 1.25}, ...]}
// Unknown members are ignored, so later versions may add fields; a missing "format" or a wrong version rejects
// the file.
#include "molc_tune.h"

#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <utility>

#include <sys/stat.h>
#include <unistd.h>

namespace molc {
namespace {

// ---- JSON values and a recursive-descent reader (RFC 8259 grammar; \u escapes outside ASCII read as '?')
struct JVal {
  enum Kind { Null, Bool, Num, Str, Arr, Obj } kind = Null;
  bool b = false;
  double num = 0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal *get(const char *name) const {
    for (const auto &kv : obj)
      if (kv.first == name) return &kv.second;
    return nullptr;
  }
};

class Reader {
 public:
  explicit Reader(const std::string &s) : s_(s) {}
  bool parse(JVal &v, std::string &why) {
    if (!value(v, 0)) {
      why = err_.empty() ? "malformed JSON" : err_;
      return false;
    }
    ws();
    if (i_ != s_.size()) {
      why = "trailing characters after the JSON value";
      return false;
    }
    return true;
  }

 private:
  const std::string &s_;
  size_t i_ = 0;
  std::string err_;

  void ws() {
    while (i_ < s_.size() && (s_[i_] == ' ' || s_[i_] == '\t' || s_[i_] == '\n' || s_[i_] == '\r')) ++i_;
  }
  bool fail(const char *what) {
    if (err_.empty()) err_ = std::string(what) + " at byte " + std::to_string(i_);
    return false;
  }
  bool lit(const char *w) {
    const size_t n = std::strlen(w);
    if (s_.compare(i_, n, w) != 0) return fail("unexpected token");
    i_ += n;
    return true;
  }
  bool value(JVal &v, int depth) {
    if (depth > 64) return fail("nesting too deep");
    ws();
    if (i_ >= s_.size()) return fail("unexpected end");
    const char c = s_[i_];
    if (c == '{') return object(v, depth);
    if (c == '[') return array(v, depth);
    if (c == '"') {
      v.kind = JVal::Str;
      return string(v.str);
    }
    if (c == 't') {
      v.kind = JVal::Bool;
      v.b = true;
      return lit("true");
    }
    if (c == 'f') {
      v.kind = JVal::Bool;
      v.b = false;
      return lit("false");
    }
    if (c == 'n') {
      v.kind = JVal::Null;
      return lit("null");
    }
    return number(v);
  }
  bool number(JVal &v) {
    const size_t i0 = i_;
    if (i_ < s_.size() && s_[i_] == '-') ++i_;
    auto digits = [&]() {
      const size_t d0 = i_;
      while (i_ < s_.size() && s_[i_] >= '0' && s_[i_] <= '9') ++i_;
      return i_ > d0;
    };
    if (!digits()) return fail("bad number");
    if (i_ < s_.size() && s_[i_] == '.') {
      ++i_;
      if (!digits()) return fail("bad number");
    }
    if (i_ < s_.size() && (s_[i_] == 'e' || s_[i_] == 'E')) {
      ++i_;
      if (i_ < s_.size() && (s_[i_] == '+' || s_[i_] == '-')) ++i_;
      if (!digits()) return fail("bad number");
    }
    v.kind = JVal::Num;
    v.num = std::strtod(s_.substr(i0, i_ - i0).c_str(), nullptr);
    return std::isfinite(v.num) || fail("number out of range");
  }
  bool hex4(unsigned &u) {
    if (i_ + 4 > s_.size()) return fail("bad \\u escape");
    u = 0;
    for (int k = 0; k < 4; ++k) {
      const char h = s_[i_++];
      u <<= 4;
      if (h >= '0' && h <= '9') u |= (unsigned)(h - '0');
      else if (h >= 'a' && h <= 'f') u |= (unsigned)(h - 'a' + 10);
      else if (h >= 'A' && h <= 'F') u |= (unsigned)(h - 'A' + 10);
      else return fail("bad \\u escape");
    }
    return true;
  }
  bool string(std::string &out) {
    ++i_;   // opening quote
    out.clear();
    while (i_ < s_.size()) {
      const char c = s_[i_++];
      if (c == '"') return true;
      if ((unsigned char)c < 0x20) return fail("control character in string");
      if (c != '\\') {
        out += c;
        continue;
      }
      if (i_ >= s_.size()) break;
      const char e = s_[i_++];
      switch (e) {
        case '"': out += '"'; break;
        case '\\': out += '\\'; break;
        case '/': out += '/'; break;
        case 'b': out += '\b'; break;
        case 'f': out += '\f'; break;
        case 'n': out += '\n'; break;
        case 'r': out += '\r'; break;
        case 't': out += '\t'; break;
        case 'u': {
          unsigned u = 0;
          if (!hex4(u)) return false;
          out += u < 0x80 ? (char)u : '?';
          break;
        }
        default: return fail("bad escape");
      }
    }
    return fail("unterminated string");
  }
  bool array(JVal &v, int depth) {
    ++i_;
    v.kind = JVal::Arr;
    ws();
    if (i_ < s_.size() && s_[i_] == ']') {
      ++i_;
      return true;
    }
    while (true) {
      v.arr.emplace_back();
      if (!value(v.arr.back(), depth + 1)) return false;
      ws();
      if (i_ >= s_.size()) return fail("unterminated array");
      if (s_[i_] == ',') {
        ++i_;
        continue;
      }
      if (s_[i_] == ']') {
        ++i_;
        return true;
      }
      return fail("expected , or ] in array");
    }
  }
  bool object(JVal &v, int depth) {
    ++i_;
    v.kind = JVal::Obj;
    ws();
    if (i_ < s_.size() && s_[i_] == '}') {
      ++i_;
      return true;
    }
    while (true) {
      ws();
      if (i_ >= s_.size() || s_[i_] != '"') return fail("expected a member name");
      std::string name;
      if (!string(name)) return false;
      ws();
      if (i_ >= s_.size() || s_[i_] != ':') return fail("expected :");
      ++i_;
      v.obj.emplace_back(std::move(name), JVal{});
      if (!value(v.obj.back().second, depth + 1)) return false;
      ws();
      if (i_ >= s_.size()) return fail("unterminated object");
      if (s_[i_] == ',') {
        ++i_;
        continue;
      }
      if (s_[i_] == '}') {
        ++i_;
        return true;
      }
      return fail("expected , or } in object");
    }
  }
};

void put_string(std::ostringstream &o, const std::string &s) {
  o << '"';
  for (const char c : s) {
    if (c == '"' || c == '\\') {
      o << '\\' << c;
    } else if ((unsigned char)c < 0x20) {
      char buf[8];
      std::snprintf(buf, sizeof buf, "\\u%04x", (unsigned)(unsigned char)c);
      o << buf;
    } else {
      o << c;
    }
  }
  o << '"';
}

constexpr const char *kFormat = "molc-tune-cache";
constexpr int kVersion = 1;

}  // namespace

bool tune_parse(const std::string &text, std::vector<TuneRecord> &out, std::string &why) {
  out.clear();
  JVal root;
  if (!Reader(text).parse(root, why)) return false;
  const JVal *fmt = root.kind == JVal::Obj ? root.get("format") : nullptr;
  if (!fmt || fmt->kind != JVal::Str || fmt->str != kFormat) {
    why = "not a molc tuning cache (no \"format\": \"molc-tune-cache\")";
    return false;
  }
  const JVal *ver = root.get("version");
  if (!ver || ver->kind != JVal::Num || ver->num != kVersion) {
    why = "unsupported tuning cache version";
    return false;
  }
  const JVal *ent = root.get("entries");
  if (!ent || ent->kind != JVal::Arr) {
    why = "tuning cache without an \"entries\" array";
    return false;
  }
  for (size_t k = 0; k < ent->arr.size(); ++k) {
    const JVal &e = ent->arr[k];
    TuneRecord r;
    auto str = [&](const char *name, std::string &dst) {
      const JVal *v = e.kind == JVal::Obj ? e.get(name) : nullptr;
      if (!v || v->kind != JVal::Str) return false;
      dst = v->str;
      return true;
    };
    auto num = [&](const char *name, double lo, double hi, double &dst) {
      const JVal *v = e.kind == JVal::Obj ? e.get(name) : nullptr;
      if (!v) return true;   // optional: stays at its default
      if (v->kind != JVal::Num || !(v->num >= lo && v->num <= hi)) return false;
      dst = v->num;
      return true;
    };
    double depth = 0, tc = 0, tg = 0, bt = 0, ms = 0;
    const bool ok = str("key", r.key) && str("device", r.device) && str("build", r.build) &&
                    num("sweep_depth", 0, 64, depth) && num("tile_cells", 0, 1 << 20, tc) &&
                    num("tile_groups", 0, 4096, tg) && num("block_threads", 0, 1024, bt) && num("best_ms", 0, 1e12, ms);
    if (!ok || depth != std::floor(depth) || tc != std::floor(tc) || tg != std::floor(tg) || bt != std::floor(bt)) {
      why = "tuning cache entry " + std::to_string(k) + " is malformed";
      out.clear();
      return false;
    }
    r.sweep_depth = (int)depth;
    r.tile_cells = (int)tc;
    r.tile_groups = (int)tg;
    r.block_threads = (int)bt;
    r.best_ms = ms;
    out.push_back(std::move(r));
  }
  return true;
}

std::string tune_serialize(const std::vector<TuneRecord> &recs) {
  std::ostringstream o;
  o << "{\"format\": \"" << kFormat << "\", \"version\": " << kVersion << ",\n \"entries\": [";
  for (size_t k = 0; k < recs.size(); ++k) {
    const TuneRecord &r = recs[k];
    char ms[40];
    std::snprintf(ms, sizeof ms, "%.6g", r.best_ms);
    o << (k ? ",\n  " : "\n  ") << "{\"key\": ";
    put_string(o, r.key);
    o << ", \"device\": ";
    put_string(o, r.device);
    o << ", \"build\": ";
    put_string(o, r.build);
    o << ", \"sweep_depth\": " << r.sweep_depth << ", \"tile_cells\": " << r.tile_cells
      << ", \"tile_groups\": " << r.tile_groups << ", \"block_threads\": " << r.block_threads
      << ", \"best_ms\": " << ms << "}";
  }
  o << (recs.empty() ? "]}\n" : "\n ]}\n");
  return o.str();
}

namespace {
std::mutex g_tune_mu;
std::string g_tune_path;                 // empty: no cache
std::vector<TuneRecord> g_tune_recs;

// Read a cache file: true with its records (none for a missing file), false with the reason.
bool read_cache(const std::string &path, std::vector<TuneRecord> &recs, std::string &why) {
  recs.clear();
  struct stat sb;
  if (stat(path.c_str(), &sb) != 0) {
    if (errno == ENOENT) return true;   // no file yet: an empty cache
    why = "cannot read " + path + ": " + std::strerror(errno);
    return false;
  }
  std::ifstream f(path, std::ios::binary);
  if (!f) {
    why = "cannot read " + path;
    return false;
  }
  std::stringstream ss;
  ss << f.rdbuf();
  if (!tune_parse(ss.str(), recs, why)) {
    why = path + ": " + why;
    return false;
  }
  return true;
}

bool same_target(const TuneRecord &a, const TuneRecord &b) {
  return a.key == b.key && a.device == b.device && a.build == b.build;
}
}  // namespace

int tune_cache_set(const char *path, std::string &why) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!path || !*path) {
    g_tune_path.clear();
    g_tune_recs.clear();
    return 0;
  }
  std::vector<TuneRecord> recs;
  if (!read_cache(path, recs, why)) return -1;
  g_tune_path = path;
  g_tune_recs = std::move(recs);
  return (int)g_tune_recs.size();
}

bool tune_cache_enabled() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return !g_tune_path.empty();
}

bool tune_cache_lookup(const std::string &key, const std::string &device, const std::string &build, TuneRecord &out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneRecord want;
  want.key = key;
  want.device = device;
  want.build = build;
  for (const TuneRecord &r : g_tune_recs)
    if (same_target(r, want)) {
      out = r;
      return true;
    }
  return false;
}

bool tune_cache_store(const TuneRecord &rec, std::string &why) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune_path.empty()) return true;
  std::vector<TuneRecord> recs;
  if (!read_cache(g_tune_path, recs, why)) recs = g_tune_recs;   // unreadable now: keep what was read before
  bool replaced = false;
  for (TuneRecord &r : recs)
    if (same_target(r, rec)) {
      r = rec;
      replaced = true;
    }
  if (!replaced) recs.push_back(rec);
  const std::string tmp = g_tune_path + ".tmp." + std::to_string((long)getpid());
  {
    std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
    if (!f) {
      why = "cannot write " + tmp + ": " + std::strerror(errno);
      return false;
    }
    f << tune_serialize(recs);
    if (!f.flush()) {
      why = "cannot write " + tmp;
      std::remove(tmp.c_str());
      return false;
    }
  }
  if (std::rename(tmp.c_str(), g_tune_path.c_str()) != 0) {
    why = "cannot replace " + g_tune_path + ": " + std::strerror(errno);
    std::remove(tmp.c_str());
    return false;
  }
  g_tune_recs = std::move(recs);
  return true;
}

}  // namespace molc
