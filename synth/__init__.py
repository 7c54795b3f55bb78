"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library's tests and benchmark.

Fields, fitted INR weights, random boxes and cell lists.  Nothing here computes any step of the
extraction method; both sides take these arrays as inputs.
"""
from . import fields, inr, boxes  # noqa: F401
