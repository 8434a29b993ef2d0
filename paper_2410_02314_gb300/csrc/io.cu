// Stack reader: one host thread per open stack reads raw uint16 frames ahead into a ring of
// (pinned, when a CUDA device is present) host buffers; the consumer takes batches in file
// order and hands each buffer back after its copy to the device has completed.  This is the
// "preload images ahead of inference" half of the paper's inference frame (Sec. 2.2).
#include <cuda_runtime.h>
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cerrno>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/sml_io.h"

struct sml_reader {
  int fd = -1;
  long long offset = 0;
  int T = 0, H = 0, W = 0, batch = 0, nbuf = 0;
  long long nbatches = 0;
  size_t frame_bytes = 0;
  std::vector<uint16_t*> bufs;
  bool pinned = false;
  // batch b lives in buffer b % nbuf; filled[k] = the batch index buffer k holds (-1: none)
  std::vector<long long> filled;
  long long next_out = 0;      // next batch to hand out
  long long next_release = 0;  // next batch to be released
  int error = 0;
  bool stop = false;
  double bytes = 0.0, read_s = 0.0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
};

namespace {

int frames_in(const sml_reader* r, long long b) {
  const long long first = b * r->batch;
  const long long n = r->T - first;
  return (int)(n < r->batch ? n : r->batch);
}

bool read_fully(int fd, void* dst, size_t n, long long off) {
  uint8_t* p = static_cast<uint8_t*>(dst);
  while (n > 0) {
    const ssize_t got = pread(fd, p, n, (off_t)off);
    if (got < 0 && errno == EINTR) continue;
    if (got <= 0) return false;
    p += got;
    n -= (size_t)got;
    off += got;
  }
  return true;
}

void reader_loop(sml_reader* r) {
  for (long long b = 0; b < r->nbatches; ++b) {
    const int k = (int)(b % r->nbuf);
    {
      std::unique_lock<std::mutex> lk(r->mu);
      // the buffer is free once the batch that used it before (b - nbuf) was released
      r->cv.wait(lk, [&] { return r->stop || r->next_release >= b - r->nbuf + 1; });
      if (r->stop) return;
    }
    const size_t n = (size_t)frames_in(r, b) * r->frame_bytes;
    const auto t0 = std::chrono::steady_clock::now();
    const bool ok = read_fully(r->fd, r->bufs[k], n, r->offset + b * (long long)r->batch * (long long)r->frame_bytes);
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    {
      std::lock_guard<std::mutex> lk(r->mu);
      r->read_s += dt;
      if (!ok) {
        r->error = SML_ERR_BAD_ARG;
        r->cv.notify_all();
        return;
      }
      r->bytes += (double)n;
      r->filled[k] = b;
    }
    r->cv.notify_all();
  }
}

void free_buffers(sml_reader* r) {
  for (uint16_t* p : r->bufs) {
    if (!p) continue;
    if (r->pinned)
      cudaFreeHost(p);
    else
      free(p);
  }
  r->bufs.clear();
}

}  // namespace

extern "C" {

int sml_reader_open(const char* path, long long offset, int T, int H, int W, int batch, int n_buffers,
                    sml_reader** out) {
  if (!path || !out || offset < 0 || T < 1 || H < 1 || W < 1 || H > 16384 || W > 16384 || batch < 1 ||
      n_buffers < 2 || n_buffers > 16)
    return SML_ERR_BAD_ARG;
  *out = nullptr;
  const int fd = open(path, O_RDONLY);
  if (fd < 0) return SML_ERR_BAD_ARG;
  struct stat sb;
  const long long need = offset + (long long)T * H * W * 2;
  if (fstat(fd, &sb) != 0 || (long long)sb.st_size < need) {
    close(fd);
    return SML_ERR_BAD_ARG;
  }
  sml_reader* r = new sml_reader();
  r->fd = fd;
  r->offset = offset;
  r->T = T;
  r->H = H;
  r->W = W;
  r->batch = batch;
  r->nbuf = n_buffers;
  r->nbatches = (T + batch - 1) / batch;
  r->frame_bytes = (size_t)H * W * sizeof(uint16_t);
  r->filled.assign(n_buffers, -1);
  const size_t bytes = (size_t)batch * r->frame_bytes;
  int ndev = 0;
  r->pinned = cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0;
  if (!r->pinned) cudaGetLastError();
  for (int k = 0; k < n_buffers; ++k) {
    void* p = nullptr;
    if (r->pinned) {
      if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) p = nullptr;
    } else if (posix_memalign(&p, 4096, bytes) != 0) {
      p = nullptr;
    }
    if (!p) {
      r->bufs.push_back(nullptr);
      free_buffers(r);
      close(fd);
      delete r;
      return SML_ERR_OOM;
    }
    r->bufs.push_back(static_cast<uint16_t*>(p));
  }
  r->th = std::thread(reader_loop, r);
  *out = r;
  return SML_OK;
}

int sml_reader_next(sml_reader* r, const uint16_t** frames, int* n_frames, long long* first_frame, int timeout_ms) {
  if (!r || !frames || !n_frames || !first_frame || timeout_ms < 0) return SML_ERR_BAD_ARG;
  std::unique_lock<std::mutex> lk(r->mu);
  const long long b = r->next_out;
  if (b >= r->nbatches) {
    *frames = nullptr;
    *n_frames = 0;
    *first_frame = r->T;
    return SML_OK;
  }
  const int k = (int)(b % r->nbuf);
  const bool got = r->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                  [&] { return r->error != 0 || r->filled[k] == b; });
  if (r->filled[k] != b) return r->error ? r->error : SML_ERR_CUDA;
  (void)got;
  *frames = r->bufs[k];
  *n_frames = frames_in(r, b);
  *first_frame = b * r->batch;
  ++r->next_out;
  return SML_OK;
}

int sml_reader_release(sml_reader* r, const uint16_t* frames) {
  if (!r || !frames) return SML_ERR_BAD_ARG;
  {
    std::lock_guard<std::mutex> lk(r->mu);
    const long long b = r->next_release;
    if (b >= r->next_out || r->bufs[b % r->nbuf] != frames) return SML_ERR_BAD_ARG;  // out of order
    r->filled[b % r->nbuf] = -1;
    ++r->next_release;
  }
  r->cv.notify_all();
  return SML_OK;
}

int sml_reader_stats(const sml_reader* r, sml_io_stats* out) {
  if (!r || !out) return SML_ERR_BAD_ARG;
  sml_reader* m = const_cast<sml_reader*>(r);
  std::lock_guard<std::mutex> lk(m->mu);
  out->bytes_read = r->bytes;
  out->read_seconds = r->read_s;
  out->wall_seconds = 0.0;
  out->frames = 0;
  return SML_OK;
}

void sml_reader_close(sml_reader* r) {
  if (!r) return;
  {
    std::lock_guard<std::mutex> lk(r->mu);
    r->stop = true;
  }
  r->cv.notify_all();
  if (r->th.joinable()) r->th.join();
  free_buffers(r);
  if (r->fd >= 0) close(r->fd);
  delete r;
}

}  // extern "C"
