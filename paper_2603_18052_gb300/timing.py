"""The three GPU timing models of Sec. 3.4 (Eq. 7-9), in ns per state-step.

A propagation call advances b states of n = d^2 complex128 values by one
step with one n x n propagator P.  The models add, from the inside out:

  kernel-only  (Eq. 7): T_k = (t_launch + 16 n^2 b / B_dev) / b
  resident P   (Eq. 8): T_r = T_k + (t_h2d(16 n b) + t_d2h(16 n b) + t_sync) / b
  host-visible (Eq. 9): T_h = T_r + (t_h2d(16 n^2) + t_alloc) / b

with t_x(m) = t_lat + m / B_inf the cost of an m-byte transfer.  Eq. 7
streams P once per state (16 n^2 bytes, no reuse across the batch), at the
best coalesced rate B_dev the device probe reached.

Readings of the constants (Table tab:probes_gpu, Sec. 3.6), chosen because
they reproduce every idealized entry of Table tab:cost_model_gpu from the
printed probe values to within the rounding of those values:
  * B_dev is the larger of the two coalesced-stream rates;
  * t_sync is the launch + synchronise time of the probe;
  * t_lat is the printed copy latency, for both directions;
  * t_alloc is the stated 3 us per cudaMalloc or cudaFree times the number of
    such calls (six in the paper's host-visible call).
"""

from dataclasses import dataclass


@dataclass
class Probes:
    """Device-probe constants (Table tab:probes_gpu): microseconds and GB/s
    (1 GB/s = 1 byte/ns)."""

    launch_us: float
    launch_sync_us: float
    lat_h2d_us: float
    lat_d2h_us: float
    h2d_gbs: float
    d2h_gbs: float
    stream_gbs: float
    alloc_calls: int = 6
    alloc_us_each: float = 3.0


def transfer_ns(m_bytes, lat_us, gbs):
    """t_x(m) = t_lat + m / B_inf in ns."""
    return lat_us * 1e3 + m_bytes / gbs


def cost_kernel(n, b, p):
    """Eq. 7: kernel-only ns per state-step."""
    return (p.launch_us * 1e3 + 16.0 * n * n * b / p.stream_gbs) / b


def cost_resident(n, b, p):
    """Eq. 8: resident-P ns per state-step."""
    x = 16.0 * n * b
    return cost_kernel(n, b, p) + (transfer_ns(x, p.lat_h2d_us, p.h2d_gbs) + transfer_ns(x, p.lat_d2h_us, p.d2h_gbs)
                                   + p.launch_sync_us * 1e3) / b


def cost_host(n, b, p):
    """Eq. 9: host-visible ns per state-step."""
    return cost_resident(n, b, p) + (transfer_ns(16.0 * n * n, p.lat_h2d_us, p.h2d_gbs)
                                     + p.alloc_calls * p.alloc_us_each * 1e3) / b


MODELS = (("kernel", cost_kernel), ("resident", cost_resident), ("host", cost_host))


def fpga_cycles(n, k=1, nsteps=1):
    """Eq. eq:cost_fpga: n^2/k + n + 4 cycles per step of Algorithm alg:fpga,
    N steps plus one start cycle."""
    return nsteps * (n * n // k + n + 4) + 1
