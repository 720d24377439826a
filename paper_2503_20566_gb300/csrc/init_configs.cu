// Starting configurations (Sec. S-2, "Configuration sampling"): a Gauss-law
// solution on the comb tree for the chain's occupations, then plaquette
// powers P_j^{t_j}.  One thread per chain.
#include "launch.h"

namespace gcf {

__global__ void k_init_configs(int N, int Lx, int Ly, int matter, const int* Q, int n_chains,
                               const int8_t* occ, const int8_t* powers, int8_t* configs,
                               int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  const int n_h = Ly * (Lx - 1), n_v = (Ly - 1) * Lx, n_s = Lx * Ly;
  const int cfg_len = n_h + n_v + n_s;
  int8_t* cfg = configs + (long long)c * cfg_len;
  for (int i = 0; i < cfg_len; ++i) cfg[i] = 0;
  int tot = 0;
  for (int s = 0; s < n_s; ++s) {
    const int p = (matter && occ) ? occ[(long long)c * n_s + s] : 0;
    cfg[n_h + n_v + s] = (int8_t)p;
    tot += p - Q[s];
  }
  if (((tot % N) + N) % N != 0) {
    atomicAdd(&status[0], 1);
    return;
  }
  auto P = [&](int x, int y) { return (int)cfg[n_h + n_v + y * Lx + x]; };
  auto H = [&](int x, int y) -> int8_t& { return cfg[y * (Lx - 1) + x]; };
  auto V = [&](int x, int y) -> int8_t& { return cfg[n_h + y * Lx + x]; };
  // rows, from the right: p + n_l - n_r = Q at (x, y), x >= 1
  for (int y = 0; y < Ly; ++y) {
    int nr = 0;
    for (int x = Lx - 1; x >= 1; --x) {
      const int nl = (((Q[y * Lx + x] - P(x, y) + nr) % N) + N) % N;
      H(x - 1, y) = (int8_t)nl;
      nr = nl;
    }
  }
  // column 0, from the top: p + n_d - n_r - n_u = Q at (0, y)
  int nu = 0;
  for (int y = Ly - 1; y >= 1; --y) {
    const int nr = H(0, y);
    const int nd = (((Q[y * Lx] - P(0, y) + nr + nu) % N) + N) % N;
    V(0, y - 1) = (int8_t)nd;
    nu = nd;
  }
  if (powers) {
    const int np = (Lx - 1) * (Ly - 1);
    for (int y = 0; y < Ly - 1; ++y)
      for (int x = 0; x < Lx - 1; ++x) {
        const int t = ((powers[(long long)c * np + y * (Lx - 1) + x] % N) + N) % N;
        if (!t) continue;
        H(x, y) = (int8_t)((H(x, y) + t) % N);
        V(x + 1, y) = (int8_t)((V(x + 1, y) + t) % N);
        H(x, y + 1) = (int8_t)((H(x, y + 1) - t + N) % N);
        V(x, y) = (int8_t)((V(x, y) - t + N) % N);
      }
  }
}

cudaError_t launch_init_configs(int N, int Lx, int Ly, int matter, const int* Q, int n_chains,
                                const int8_t* occ, const int8_t* powers, int8_t* configs,
                                int* status, cudaStream_t st) {
  k_init_configs<<<(n_chains + 127) / 128, 128, 0, st>>>(N, Lx, Ly, matter, Q, n_chains, occ, powers,
                                                          configs, status);
  return cudaGetLastError();
}

}  // namespace gcf
