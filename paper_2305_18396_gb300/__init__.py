"""GB300 library for the server-side homomorphic matrix product of
"LLMs Can Understand Encrypted Prompt" (Algorithm 1, Sec. 3.1.1).

The CUDA library (csrc/, built into _lib/libhe_gb300.so) implements the C ABI
of include/he_gb300.h; ``binding`` is its thin ctypes binding and
``workloads`` describes the BERT-shaped products the benchmark runs.  Importing
the package does not load the library; ``binding`` raises if it is missing.
"""
__all__ = ["binding", "build", "params", "synthetic", "workloads"]
