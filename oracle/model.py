"""Execution-model closed forms of the paper (Section 4), test infrastructure.

Symbols follow Table 1: ``n`` = N_process, ``t_init`` = T_init,
``t_ctx`` = T_ctx_switch, ``t_in`` = T_data_in, ``t_out`` = T_data_out,
``t_comp`` = T_comp. All times share one unit.

Readings where the paper is silent or garbled (each also listed in the
design notes):

* The class rule (Section 4.2.3) defines compute-intensive as
  T_in <= T_comp and T_out <= T_comp, and I/O-intensive as both larger than
  T_comp; a task with only one of them larger is what Section 6 calls
  "intermediate" (matrix multiply). ``classify`` returns that third class and
  ``shared_time`` charges it with I/O-intensive style (Eq. 7), the policy for
  tasks whose copies are not covered by compute.
* Eq. 2 assumes every kernel overlaps completely and that copies in opposite
  directions do not overlap (Section 4.2.3). ``shared_time_duplex`` is an
  added variant for a link that carries both directions at once and for
  kernels that need more than one wave of the GPU: the longer of the
  pipeline's copy chain (Eq. 7's form) and its compute chain.
"""
from __future__ import annotations


def t_total_no_vt(n, t_init, t_in, t_comp, t_out, t_ctx):
    """Eq. 1: N processes run one after another, each paying T_init, with a
    context switch between consecutive processes."""
    return n * (t_init + t_in + t_comp + t_out) + (n - 1) * t_ctx


def t_total_ci_ps1(n, t_in, t_comp, t_out):
    """Eq. 2: compute-intensive tasks issued in programming style 1 (all
    inputs, then all kernels, then all outputs): the copies of all processes
    serialise, the kernels overlap into one T_comp."""
    return n * (t_in + t_out) + t_comp


def t_total_ci_ps2(n, t_in, t_comp, t_out):
    """Eq. 3: compute-intensive tasks in programming style 2 (per stream:
    input, kernel, output): kernels serialise, one input and one output copy
    stay exposed."""
    return t_in + n * t_comp + t_out


def t_total_ioi_ps1(n, t_in, t_comp, t_out):
    """Eq. 4: I/O-intensive tasks in style 1 -- the same expression as Eq. 2."""
    return n * (t_in + t_out) + t_comp


def t_total_ioi_ps2_piecewise(n, t_in, t_comp, t_out):
    """Eqs. 5 and 6: I/O-intensive tasks in style 2, by which copy is longer."""
    if t_out < t_in:
        return n * t_in + t_comp + t_out  # Eq. 5
    return t_in + t_comp + n * t_out  # Eq. 6


def t_total_ioi_ps2(n, t_in, t_comp, t_out):
    """Eq. 7: Eqs. 5 and 6 in one expression with max and min."""
    return n * max(t_in, t_out) + t_comp + min(t_in, t_out)


def speedup_ci(n, t_init, t_in, t_comp, t_out, t_ctx):
    """Eq. 8: Eq. 1 over Eq. 2."""
    return t_total_no_vt(n, t_init, t_in, t_comp, t_out, t_ctx) / t_total_ci_ps1(n, t_in, t_comp, t_out)


def speedup_ioi(n, t_init, t_in, t_comp, t_out, t_ctx):
    """Eq. 9: Eq. 1 over Eq. 7."""
    return t_total_no_vt(n, t_init, t_in, t_comp, t_out, t_ctx) / t_total_ioi_ps2(n, t_in, t_comp, t_out)


def speedup_max_ci(t_init, t_in, t_comp, t_out, t_ctx):
    """Eq. 10: the limit of Eq. 8 as N grows without bound."""
    return (t_init + t_in + t_comp + t_out + t_ctx) / (t_in + t_out)


def speedup_max_ioi(t_init, t_in, t_comp, t_out, t_ctx):
    """Eq. 11: the limit of Eq. 9 as N grows without bound."""
    return (t_init + t_in + t_comp + t_out + t_ctx) / max(t_in, t_out)


CI, IOI, INTERMEDIATE = "C-I", "IO-I", "intermediate"


def classify(t_in, t_comp, t_out):
    """Task class of Section 4.2.3 (third class: see the module docstring)."""
    if t_in <= t_comp and t_out <= t_comp:
        return CI
    if t_in > t_comp and t_out > t_comp:
        return IOI
    return INTERMEDIATE


def shared_time(n, t_in, t_comp, t_out):
    """Predicted shared time under the paper's policy (Section 4.2.3 and
    Section 5): style 1 and Eq. 2 for compute-intensive tasks, style 2 and
    Eq. 7 otherwise."""
    if classify(t_in, t_comp, t_out) == CI:
        return t_total_ci_ps1(n, t_in, t_comp, t_out)
    return t_total_ioi_ps2(n, t_in, t_comp, t_out)


def shared_time_duplex(n, t_in, t_comp_wave, t_out, waves):
    """Variant of Eq. 7 for a host link that carries both directions at once
    and for a compute phase that needs ``waves`` waves of the GPU.

    Each task runs input copy, kernel, output copy; input copies of different
    tasks share one direction of the link, output copies the other, and the
    kernels of different tasks run side by side, ``t_comp_wave`` per wave.
    The shared time is the longer of two chains of that pipeline:

    * the copy chain: the longer direction streams all N copies, with one
      task's kernel and one copy of the shorter direction exposed at the ends,
      ``n max(t_in, t_out) + t_comp_wave + min(t_in, t_out)`` (Eq. 7's form);
    * the compute chain: the first input, every wave, the last output,
      ``t_in + waves t_comp_wave + t_out``.

    Neither chain can be shortened, so the value is a lower bound on the
    pipeline's makespan; with one wave it is the makespan itself, and equals
    Eq. 7. At N = 1 with one wave it is T_in + T_comp + T_out.
    """
    if n <= 0:
        return 0.0
    copy_chain = n * max(t_in, t_out) + t_comp_wave + min(t_in, t_out)
    compute_chain = t_in + waves * t_comp_wave + t_out
    return max(copy_chain, compute_chain)


def waves(n_tasks, ctas_per_task, sms, ctas_per_sm):
    """Number of full-GPU waves for n_tasks kernels of ctas_per_task blocks,
    with ``sms * ctas_per_sm`` blocks resident at once: the ceiling of blocks
    over slots (0 for no tasks)."""
    if sms <= 0 or ctas_per_sm <= 0:
        raise ValueError("waves: no block slots")
    blocks = n_tasks * ctas_per_task
    slots = sms * ctas_per_sm
    return (blocks + slots - 1) // slots


def deviation(measured, predicted):
    """Relative model deviation |measured - predicted| / predicted (Section 6)."""
    return abs(measured - predicted) / predicted
