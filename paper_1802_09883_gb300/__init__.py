"""Reproducible grouped SUM (repro<T,L>) on GB300: Python binding placeholder."""
